// DST-I of the mixed path on the tcgen05 tensor cores: split-bf16 folded GEMM, FP32 accumulate.
//
// The preconditioner's transform along x (Sec. 2.4) is y = S x per row with S^2 = I.  Folding the
// input pairs (j, n-1-j) halves the work (see k_dst.cu).  Each operand value v is split into two
// bf16 numbers hi = bf16(v), lo = bf16(v - hi); the product is formed from hi*hi + hi*lo + lo*hi
// (lo*lo is below FP32 rounding of the sum), accumulated in FP32 in tensor memory.
//
// Forward (x float64 -> spectrum float32): fold on the input,
//   y[2k']   = sum_j' S[j'][2k']   u[j'],  u = x[j'] + x[n-1-j'] (middle once)   -> "parity 0"
//   y[2k'+1] = sum_j' S[j'][2k'+1] v[j'],  v = x[j'] - x[n-1-j']                 -> "parity 1"
// and the spectrum is stored parity-permuted: columns [0, ku) hold the even modes 2k', columns
// [ku, n) the odd modes 2k'+1 (the tridiagonal factors use the same column order).
// Inverse (spectrum float32 -> z float64): fold on the output,
//   E[k] = sum_j' S[2j'][k] y[2j'],  O[k] = sum_j' S[2j'+1][k] y[2j'+1],
//   z[k] = E[k] + O[k],  z[n-1-k] = E[k] - O[k]           (k < ceil(n/2); O = 0 at the middle).
//
// Data movement: a pack kernel writes the A operand (folded / split rows) as 128-row x 64-column
// bf16 tiles already in the canonical K-major 128-byte-swizzled shared-memory layout; the constant
// B operands (rows of S) are packed the same way once per plan.  The GEMM kernel then moves every
// stage with four cp.async.bulk copies (TMA engine) completing on an mbarrier, one thread issues
// tcgen05.mma from shared-memory descriptors into a 128 x 256 FP32 accumulator in tensor memory,
// tcgen05.commit releases each stage, and four warps read the accumulator with tcgen05.ld.
// Every wait is bounded: on expiry the kernel records an error code and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <atomic>
#include <cstdlib>
#include <cstdint>

#include "internal.h"

#include <utility>
#include <vector>

namespace lag {

namespace {

constexpr int TM = 128;          // rows per tile (MMA M)
constexpr int TN = 256;          // output columns per tile (MMA N)
constexpr int TK = 64;           // K per stage (one 128-byte swizzle atom of bf16)
constexpr int A_TILE = TM * TK * 2;   // 16 KB
constexpr int B_TILE = TN * TK * 2;   // 32 KB
constexpr uint32_t TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1LL << 26;

// element (r, k) of a rows x 64 tile in the K-major SWIZZLE_128B layout (byte offset)
__host__ __device__ __forceinline__ uint32_t swz(int r, int k) {
  return (uint32_t)r * 128u + ((uint32_t)((k >> 3) ^ (r & 7)) << 4) + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  __nv_bfloat16 b = __float2bfloat16_rn(f);
  return *reinterpret_cast<uint16_t *>(&b);
}

// split v into bf16 hi + bf16 lo (float64 arithmetic: used once per plan for S)
__device__ __forceinline__ void split2(double v, uint16_t &hi, uint16_t &lo) {
  const float f = (float)v;
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  const float r = (float)(v - (double)__bfloat162float(h));
  hi = *reinterpret_cast<uint16_t *>(&h);
  lo = bf16_bits(r);
}

// the same split in float32 arithmetic (per apply: FP64 throughput is 1/61 of FP32 on this part;
// hi + lo keeps 16 significant bits, far inside float32 rounding)
__device__ __forceinline__ void split2f(float f, uint16_t &hi, uint16_t &lo) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  hi = *reinterpret_cast<uint16_t *>(&h);
  lo = bf16_bits(f - __bfloat162float(h));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false when the limit expired
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 32) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
  return d;
}

// instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

// the same MMA with N = 128 (half-width tiles of the split-bf16 GEMM)
constexpr uint32_t IDESC_H = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((TN / 2) >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
__device__ __forceinline__ void mma_bf16_h(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(IDESC_H), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// 16 consecutive columns of a lane's row (fewer live registers than 32 in register-tight epilogues)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// ------------------------------------------------------------------------------ packing
// B operands, once per plan.  which: 0 fwd even (B[n][k] = S[k][2n]), 1 fwd odd (S[k][2n+1]),
// 2 inv E (S[n][2k]), 3 inv O (S[n][2k+1], zero row at n = kv for odd n).  Layout per matrix:
// [n tile][k stage][hi | lo][TN x TK swizzled].
__global__ void pack_b_kernel(const double *su, const double *sv, int ku, int kv, int nks, int nnt, uint8_t *out,
                              size_t mat_bytes) {
  const int which = blockIdx.z;
  const int n = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnt * TN || k >= nks * TK) return;
  double v = 0.0;
  switch (which) {
    case 0: if (n < ku && k < ku) v = su[(size_t)k * ku + n]; break;
    case 1: if (n < kv && k < kv) v = sv[(size_t)k * kv + n]; break;
    case 2: if (n < ku && k < ku) v = su[(size_t)n * ku + k]; break;
    default: if (n < kv && k < kv) v = sv[(size_t)n * kv + k]; break;
  }
  uint16_t hi, lo;
  split2(v, hi, lo);
  const size_t tile = (size_t)(n / TN) * nks + (k / TK);
  uint8_t *base = out + (size_t)which * mat_bytes + tile * 2 * B_TILE;
  const uint32_t off = swz(n % TN, k % TK);
  *reinterpret_cast<uint16_t *>(base + off) = hi;
  *reinterpret_cast<uint16_t *>(base + B_TILE + off) = lo;
}

// A operand of the forward transform: one thread per (row, 8 consecutive fold indices), both
// parities; layout [parity][m tile][k stage][hi | lo][TM x TK swizzled]
template <typename TI>
__global__ void __launch_bounds__(256) pack_a_fwd_kernel(const TI *__restrict__ x, int rows, int n, int ku, int kv,
                                                         int nks, int nmt, uint8_t *__restrict__ out,
                                                         const KrylovScalars *__restrict__ sc, int rpr, int rscale) {
  const int chunks = nks * (TK / 8);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;  // < nmt TM chunks, far below 2^32
  if (t >= (unsigned)(nmt * TM * chunks)) return;
  const int row = (int)(t / (unsigned)chunks), ch = (int)t - row * chunks;
  const int k0 = ch * 8;
  const bool live = row < rows && (sc == nullptr || sc[row / rpr].state == ST_RUN);
  // PCG residuals enter scaled by 2^-e (residual_exponent), undone by the inverse butterfly
  const int es = (live && rscale && sc != nullptr) ? -residual_exponent(sc, row / rpr) : 0;
  alignas(16) uint16_t uh[8], ul[8], vh[8], vl[8];
  const TI *xr = x + (size_t)(live ? row : 0) * n;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int j = k0 + e;
    float u = 0.f, w = 0.f;
    if (live) {
      // (float) (x 2^es) by integer operations on the bits (the conversion would take the FP64 pipe)
      if (j < kv) {
        const float a = narrow_pow2((double)xr[j], es), b = narrow_pow2((double)xr[n - 1 - j], es);
        u = a + b;
        w = a - b;
      } else if (j < ku) {
        u = narrow_pow2((double)xr[j], es);  // middle element of an odd-length row
      }
    }
    split2f(u, uh[e], ul[e]);
    split2f(w, vh[e], vl[e]);
  }
  const int mt = row / TM, r = row % TM, ks = k0 / TK, kk = k0 % TK;
  const uint32_t off = swz(r, kk);
  for (int par = 0; par < 2; ++par) {
    uint8_t *tile = out + (((size_t)par * nmt + mt) * nks + ks) * 2 * A_TILE;
    *reinterpret_cast<uint4 *>(tile + off) = *reinterpret_cast<const uint4 *>(par ? vh : uh);
    *reinterpret_cast<uint4 *>(tile + A_TILE + off) = *reinterpret_cast<const uint4 *>(par ? vl : ul);
  }
}

// A operand of the inverse transform from the parity-permuted spectrum (no fold)
__global__ void __launch_bounds__(256) pack_a_inv_kernel(const float *__restrict__ y, int rows, int n, int ku, int kv,
                                                         int nks, int nmt, uint8_t *__restrict__ out,
                                                         const KrylovScalars *__restrict__ sc, int rpr) {
  const int chunks = nks * (TK / 8);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;  // < nmt TM chunks, far below 2^32
  if (t >= (unsigned)(nmt * TM * chunks)) return;
  const int row = (int)(t / (unsigned)chunks), ch = (int)t - row * chunks;
  const int k0 = ch * 8;
  const bool live = row < rows && (sc == nullptr || sc[row / rpr].state == ST_RUN);
  const float *yr = y + (size_t)(live ? row : 0) * n;
  float ev[8], ov[8];
  if (live && k0 + 8 <= kv && (((size_t)row * n) & 3) == 0 && (ku & 3) == 0) {
    // whole chunks of both halves, 16-byte aligned: two float4 loads each
    const float4 *e4 = reinterpret_cast<const float4 *>(yr + k0), *o4 = reinterpret_cast<const float4 *>(yr + ku + k0);
    const float4 a = __ldg(e4), b = __ldg(e4 + 1), c = __ldg(o4), d = __ldg(o4 + 1);
    ev[0] = a.x; ev[1] = a.y; ev[2] = a.z; ev[3] = a.w; ev[4] = b.x; ev[5] = b.y; ev[6] = b.z; ev[7] = b.w;
    ov[0] = c.x; ov[1] = c.y; ov[2] = c.z; ov[3] = c.w; ov[4] = d.x; ov[5] = d.y; ov[6] = d.z; ov[7] = d.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = k0 + e;
      ev[e] = (live && j < ku) ? yr[j] : 0.f;
      ov[e] = (live && j < kv) ? yr[ku + j] : 0.f;
    }
  }
  alignas(16) uint16_t eh[8], el[8], oh[8], ol[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    split2f(ev[e], eh[e], el[e]);
    split2f(ov[e], oh[e], ol[e]);
  }
  const int mt = row / TM, r = row % TM, ks = k0 / TK, kk = k0 % TK;
  const uint32_t off = swz(r, kk);
  for (int par = 0; par < 2; ++par) {
    uint8_t *tile = out + (((size_t)par * nmt + mt) * nks + ks) * 2 * A_TILE;
    *reinterpret_cast<uint4 *>(tile + off) = *reinterpret_cast<const uint4 *>(par ? oh : eh);
    *reinterpret_cast<uint4 *>(tile + A_TILE + off) = *reinterpret_cast<const uint4 *>(par ? ol : el);
  }
}

// ------------------------------------------------------------------------------ GEMM
// Persistent, warp-specialised: grid = min(tiles, SMs), 192 threads.
//   warp 0 (one lane): producer, cp.async.bulk of the packed A / B tiles into a ring of stages;
//   warp 1 (one lane): MMA issuer, NPROD split products per 16-wide K step into one of two
//                      tensor-memory accumulators (256 columns each);
//   warps 2-5:         epilogue, tcgen05.ld of the finished accumulator (warp w reads lanes
//                      32 (w % 4) ..), stores, then hands the accumulator back.
// The stage ring runs across tile boundaries and the two accumulators let the epilogue of one
// tile overlap the main loop of the next.  Tiles are ordered (parity, m tile, n tile), n fastest,
// so consecutive tiles reuse the same A rows from L2.  NPROD = 3: hi*hi + hi*lo + lo*hi;
// NPROD = 2: hi*hi + lo*hi (B = bf16(S)); NPROD = 1: hi*hi.
// HALF: 128 x 128 tiles, each the 128-column half of a packed 256-column B tile (its first or last
// 16 KB of 128-byte rows): twice the tiles, for transforms whose 128 x 256 tiles would leave most
// SMs idle (one right-hand side: 64 tiles on 152 SMs); the stages then hold one K tile of A and
// of the two B halves, three to six of them.
template <int NPROD, bool HALF>
struct TcCfg {
  static constexpr int TNK = HALF ? TN / 2 : TN;  // output columns per tile
  static constexpr int BT = TNK * TK * 2;          // bytes of one B K tile of the tile's columns
  static constexpr int A_BYTES = (NPROD >= 2 ? 2 : 1) * A_TILE;
  static constexpr int B_BYTES = (NPROD >= 3 ? 2 : 1) * BT;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int NST = (196608 / STAGE_BYTES) < 6 ? (196608 / STAGE_BYTES) : 6;
  static constexpr int SMEM = NST * STAGE_BYTES + 1024 + 256;
};

template <int NPROD, bool HALF>
__global__ void __launch_bounds__(192, 1) dst_tc_gemm_kernel(const uint8_t *__restrict__ apack,
                                                             const uint8_t *__restrict__ bpack, size_t b_mat_bytes,
                                                             int nks, int nmt, int nnt, int rows, float *__restrict__ out,
                                                             int ld, int ku, int nvalid0, int nvalid1,
                                                             const KrylovScalars *__restrict__ sc, int rpr,
                                                             int *__restrict__ err) {
  using Cfg = TcCfg<NPROD, HALF>;
  constexpr int NST = Cfg::NST;
  constexpr int TNK = Cfg::TNK;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  const uint32_t bars = base + NST * Cfg::STAGE_BYTES;
  const uint32_t full0 = bars, empty0 = bars + 8 * NST, tfull0 = bars + 16 * NST, tempty0 = tfull0 + 16;
  volatile uint32_t *holder = reinterpret_cast<volatile uint32_t *>(gbase + NST * Cfg::STAGE_BYTES + 16 * NST + 32);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + NST * Cfg::STAGE_BYTES + 16 * NST + 40);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = 2 * nmt * nnt;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)holder)),
                 "r"(2 * TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 4);  // one arrive per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;

  // tile t -> (parity, m tile, n tile); tiles that only hold finished right-hand sides, or lie
  // beyond a parity's valid columns, are skipped by every role alike
  auto decode = [&](int t, int &par, int &mt, int &nt) {
    nt = t % nnt;
    mt = (t / nnt) % nmt;
    par = t / (nnt * nmt);
  };
  auto wanted = [&](int par, int mt, int nt) -> bool {
    if (nt * TNK >= (par ? nvalid1 : nvalid0)) return false;
    if (sc == nullptr) return true;
    const int m0 = mt * TM;
    const int r0 = m0 / rpr, r1 = (min(m0 + TM, rows) - 1) / rpr;
    for (int r = r0; r <= r1; ++r)
      if (sc[r].state == ST_RUN) return true;
    return false;
  };

  if (warp == 0) {
    if (lane == 0) {  // producer
      int it = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int par, mt, nt;
        decode(t, par, mt, nt);
        if (!wanted(par, mt, nt)) continue;
        const uint8_t *atiles = apack + ((size_t)par * nmt + mt) * nks * 2 * A_TILE;
        // packed B: [parity][256-column tile][K tile][hi, lo: 256 rows of 128 bytes each]
        const uint8_t *btiles = bpack + (size_t)par * b_mat_bytes +
                                (size_t)(HALF ? nt >> 1 : nt) * nks * 2 * B_TILE + (HALF ? (nt & 1) * Cfg::BT : 0);
        for (int kk = 0; kk < nks; ++kk, ++it) {
          const int s = it % NST, use = it / NST;
          if (it >= NST && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) {
            atomicExch(err, 1);
            *abort_flag = 1;
            break;
          }
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
          const uint32_t fb = full0 + 8 * s;
          mbar_expect_tx(fb, Cfg::STAGE_BYTES);
          bulk_g2s(st, atiles + (size_t)kk * 2 * A_TILE, Cfg::A_BYTES, fb);
          if constexpr (HALF) {  // the hi and lo halves are 32 KB apart in the packed tile
            bulk_g2s(st + Cfg::A_BYTES, btiles + (size_t)kk * 2 * B_TILE, Cfg::BT, fb);
            if (NPROD >= 3) bulk_g2s(st + Cfg::A_BYTES + Cfg::BT, btiles + (size_t)kk * 2 * B_TILE + B_TILE, Cfg::BT, fb);
          } else {
            bulk_g2s(st + Cfg::A_BYTES, btiles + (size_t)kk * 2 * B_TILE, Cfg::B_BYTES, fb);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      // stage position and phase kept incrementally, descriptors as one OR of the constant upper
      // bits with the 16-byte address (a single thread's per-stage work idles the tensor pipe)
      constexpr uint64_t DHI = ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61) | (1ull << 16);
      constexpr uint32_t ALO = A_TILE >> 4, BHI = Cfg::A_BYTES >> 4, BLO = (Cfg::A_BYTES + Cfg::BT) >> 4;
      int s = 0, tc = 0;
      uint32_t ph = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int par, mt, nt;
        decode(t, par, mt, nt);
        if (!wanted(par, mt, nt)) continue;
        const int acc = tc & 1, ause = tc >> 1;
        if (tc >= 2 && !mbar_wait(tempty0 + 8 * acc, (ause - 1) & 1)) {
          atomicExch(err, 4);
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(acc * TMEM_COLS);
        for (int kk = 0; kk < nks; ++kk) {
          if (!mbar_wait(full0 + 8 * s, ph)) {
            atomicExch(err, 2);
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = (base + s * Cfg::STAGE_BYTES) >> 4;
          const uint32_t f = kk == 0 ? 0u : 1u;
#pragma unroll
          for (int sub = 0; sub < TK / 16; ++sub) {  // 16 bf16 along K: 32 bytes, 2 units of 16
            if constexpr (HALF) {
              mma_bf16_h(d, DHI | (sa + 2 * sub), DHI | (sa + BHI + 2 * sub), sub == 0 ? f : 1u);
              if (NPROD >= 3) mma_bf16_h(d, DHI | (sa + 2 * sub), DHI | (sa + BLO + 2 * sub), 1u);
              if (NPROD >= 2) mma_bf16_h(d, DHI | (sa + ALO + 2 * sub), DHI | (sa + BHI + 2 * sub), 1u);
            } else {
              mma_bf16(d, DHI | (sa + 2 * sub), DHI | (sa + BHI + 2 * sub), sub == 0 ? f : 1u);
              if (NPROD >= 3) mma_bf16(d, DHI | (sa + 2 * sub), DHI | (sa + BLO + 2 * sub), 1u);
              if (NPROD >= 2) mma_bf16(d, DHI | (sa + ALO + 2 * sub), DHI | (sa + BHI + 2 * sub), 1u);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                       : "memory");
          if (++s == NST) {
            s = 0;
            ph ^= 1u;
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tfull0 + 8 * acc)
                     : "memory");
        ++tc;
      }
    }
  } else {  // epilogue warps 2..5: tensor-memory lanes 32 (warp % 4) ..
    const int lg = warp & 3;
    const bool vec = ((ld & 3) == 0) && ((ku & 3) == 0);
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int par, mt, nt;
      decode(t, par, mt, nt);
      if (!wanted(par, mt, nt)) continue;
      const int acc = tc & 1, ause = tc >> 1;
      const bool ok = mbar_wait(tfull0 + 8 * acc, ause & 1);
      __syncwarp();
      if (!ok) {
        if (lane == 0) atomicExch(err, 3);
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = mt * TM + lg * 32 + lane;
      const int n0 = nt * TNK;
      const int ncols = min(TNK, (par ? nvalid1 : nvalid0) - n0);
      float *orow = out + (size_t)row * ld + (size_t)par * ku + n0;
      for (int c0 = 0; c0 < TNK; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * TMEM_COLS + c0), v);
        if (row >= rows || c0 >= ncols) continue;
        if (vec && c0 + 32 <= ncols) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<float4 *>(orow + c0 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (c0 + q < ncols) orow[c0 + q] = v[q];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * acc) : "memory");
      ++tc;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS) : "memory");
}

// z[k] = E[k] + O[k], z[n-1-k] = E[k] - O[k]   (eo rows: [E (ku) | O (ku)])
__global__ void __launch_bounds__(256) butterfly_kernel(const float *__restrict__ eo, double *__restrict__ z, int rows,
                                                        int n, int ku, int kv, const KrylovScalars *__restrict__ sc,
                                                        int rpr, int rscale) {
  const int row = blockIdx.x;  // one block per row, its modes over the threads
  if (row >= rows || (sc != nullptr && sc[row / rpr].state != ST_RUN)) return;
  const float *er = eo + (size_t)row * 2 * ku;
  const int es = (rscale && sc != nullptr) ? residual_exponent(sc, row / rpr) : 0;
  double *zr = z + (size_t)row * n;
  for (int k = threadIdx.x; k < ku; k += blockDim.x) {
    double e = (double)er[k], o = (double)er[ku + k];
    if (es != 0) {
      e = scale_pow2(e, es);
      o = scale_pow2(o, es);
    }
    zr[k] = e + o;
    if (k < kv) zr[n - 1 - k] = e - o;
  }
}

// The butterfly fused with the CG update of the next step: per right-hand side (rpr rows each),
// z = butterfly(E, O), then rz_new = (r, z), zq = (z, q) and beta (Fletcher-Reeves or
// Polak-Ribiere), finished by the last block in a fixed order.  grid (blocks, nrhs).
__global__ void __launch_bounds__(256) butterfly_beta_kernel(const float *__restrict__ eo, double *__restrict__ z,
                                                             const double *__restrict__ r, const double *__restrict__ q,
                                                             int n, int ku, int kv, int rpr, int flexible,
                                                             KrylovScalars *sc, Reduce red) {
  const int rhs = blockIdx.y;
  if (sc[rhs].state != ST_RUN) return;
  const size_t row0 = (size_t)rhs * rpr;
  const int es = residual_exponent(sc, rhs);  // the forward pack scaled r by 2^-e
  double a0 = 0.0, a1 = 0.0;
  // rows round-robin over the blocks, a row's modes over the threads (no 64-bit index division);
  // E +- O in float32 (the spectrum's precision), widened with the residual's scale by integer
  // operations on the bits, the CG dots in float64
  for (int rl = blockIdx.x; rl < rpr; rl += gridDim.x) {
    const size_t row = row0 + (size_t)rl;
    const float *er = eo + row * 2 * ku;
#pragma unroll 4
    for (int k = threadIdx.x; k < ku; k += blockDim.x) {
      const float e = er[k], o = er[ku + k];
      const size_t i1 = row * n + k;
      const double z1 = widen_pow2(e + o, es);
      z[i1] = z1;
      a0 = fma(r[i1], z1, a0);
      if (flexible) a1 = fma(z1, q[i1], a1);
      if (k < kv) {
        const size_t i2 = row * n + (n - 1 - k);
        const double z2 = widen_pow2(e - o, es);
        z[i2] = z2;
        a0 = fma(r[i2], z2, a0);
        if (flexible) a1 = fma(z2, q[i2], a1);
      }
    }
  }
  double v2[2] = {a0, a1}, tot[2];
  __shared__ double sh[64];
  block_sum<2>(v2, sh);
  if (publish_partials<2>(red, rhs, blockIdx.x, gridDim.x, v2, tot)) {
    KrylovScalars &S = sc[rhs];
    const double rz_new = tot[0];
    S.zq = tot[1];
    // the first direction of a solve is z itself (beta = 0)
    S.beta = (S.iters == 0) ? 0.0 : (flexible ? (-S.alpha * tot[1] / S.rz) : (rz_new / S.rz));
    S.rz = rz_new;
    if (!isfinite(S.beta) || !isfinite(rz_new) || !isfinite(tot[1])) S.state = ST_NAN;
  }
}

// parity permutation of spectra (natural mode order <-> [even modes | odd modes])
__global__ void permute_kernel(const float *in, float *out, int rows, int n, int ku, int to_perm) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * n) return;
  const int row = (int)(t / n), c = (int)(t % n);
  const int j = (c < ku) ? 2 * c : 2 * (c - ku) + 1;  // mode stored at permuted column c
  if (to_perm) out[(size_t)row * n + c] = in[(size_t)row * n + j];
  else out[(size_t)row * n + j] = in[(size_t)row * n + c];
}

__global__ void unpermute_widen_kernel(const float *in, double *out, int rows, int n, int ku) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * n) return;
  const int row = (int)(t / n), c = (int)(t % n);
  const int j = (c < ku) ? 2 * c : 2 * (c - ku) + 1;
  out[(size_t)row * n + j] = (double)in[(size_t)row * n + c];
}

// ------------------------------------------------------------------------------ host side
static int div_up(int a, int b) { return (a + b - 1) / b; }

bool dst_tc_supported(int n) { return n >= 16; }

size_t dst_tc_bytes(int n) {
  const int ku = (n + 1) / 2;
  const int nks = div_up(ku, TK), nnt = div_up(ku, TN);
  return 4 * (size_t)nnt * nks * 2 * B_TILE;
}

void dst_build_tc(DstPlan &dp, DevBuf &store, size_t off, cudaStream_t s) {
  const int nks = div_up(dp.ku, TK), nnt = div_up(dp.ku, TN);
  dp.kpad_u = nks;  // stages along K
  dp.npad_u = nnt;  // tiles along N
  dp.tc_bmat_bytes = (size_t)nnt * nks * 2 * B_TILE;
  dp.tc_b = store.as<uint8_t>() + off;
  dim3 g(div_up(nks * TK, 128), nnt * TN, 4);
  pack_b_kernel<<<g, 128, 0, s>>>(dp.su, dp.sv, dp.ku, dp.kv, nks, nnt, dp.tc_b, dp.tc_bmat_bytes);
  count_launch();
  LAG_LAUNCH_CHECK();
}

template <int NPROD, bool HALF>
static void gemm_launch_nh(const DstPlan &dp, const uint8_t *apack, const uint8_t *bpack, int rows, float *out, int ld,
                           int nvalid0, int nvalid1, const KrylovScalars *sc, int rpr, int *err, cudaStream_t s) {
  static PerDeviceOnce attr;
  attr.run([] {
    LAG_CUDA_CHECK(cudaFuncSetAttribute(dst_tc_gemm_kernel<NPROD, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        TcCfg<NPROD, HALF>::SMEM));
  });
  const int nks = dp.kpad_u, nnt = dp.npad_u * (HALF ? 2 : 1), nmt = div_up(rows, TM);
  const int ntiles = 2 * nmt * nnt;
  const int grid = std::min(ntiles, 152);
  dst_tc_gemm_kernel<NPROD, HALF><<<grid, 192, TcCfg<NPROD, HALF>::SMEM, s>>>(
      apack, bpack, dp.tc_bmat_bytes, nks, nmt, nnt, rows, out, ld, dp.ku, nvalid0, nvalid1, sc, rpr, err);
}
static int device_sms();
// 128 x 256 tiles unless they would leave more than half the SMs idle (then 128 x 128 tiles)
template <int NPROD>
static void gemm_launch_n(const DstPlan &dp, const uint8_t *apack, const uint8_t *bpack, int rows, float *out, int ld,
                          int nvalid0, int nvalid1, const KrylovScalars *sc, int rpr, int *err, cudaStream_t s) {
  const int tiles = 2 * div_up(rows, TM) * dp.npad_u;
  if (2 * tiles <= device_sms())
    gemm_launch_nh<NPROD, true>(dp, apack, bpack, rows, out, ld, nvalid0, nvalid1, sc, rpr, err, s);
  else
    gemm_launch_nh<NPROD, false>(dp, apack, bpack, rows, out, ld, nvalid0, nvalid1, sc, rpr, err, s);
}

static void gemm_launch(const DstPlan &dp, const uint8_t *apack, const uint8_t *bpack, int rows, float *out, int ld,
                        int nvalid0, int nvalid1, const KrylovScalars *sc, int rpr, int *err, cudaStream_t s) {
  switch (dp.tc_products) {
    case 1: gemm_launch_n<1>(dp, apack, bpack, rows, out, ld, nvalid0, nvalid1, sc, rpr, err, s); break;
    case 2: gemm_launch_n<2>(dp, apack, bpack, rows, out, ld, nvalid0, nvalid1, sc, rpr, err, s); break;
    default: gemm_launch_n<3>(dp, apack, bpack, rows, out, ld, nvalid0, nvalid1, sc, rpr, err, s); break;
  }
  count_launch();
  LAG_LAUNCH_CHECK();
}

size_t dst_tc_scratch_bytes(const DstPlan &dp, int rows) {
  const size_t nmt = div_up(rows, TM);
  return 2 * nmt * dp.kpad_u * 2 * A_TILE + (size_t)rows * 2 * dp.ku * sizeof(float) + 256;
}

void dst_apply_tc_d2f(const DstPlan &dp, const double *x, float *y, int rows, int rpr, const KrylovScalars *sc,
                      cudaStream_t s, bool rscale) {
  if (rows <= 0) return;
  uint8_t *apack = dp.tc_scratch;
  const int nks = dp.kpad_u, nmt = div_up(rows, TM);
  {
    ProfScope prof(KC_DSTTC_FWD, s);
    const long long threads = (long long)nmt * TM * nks * (TK / 8);
    pack_a_fwd_kernel<double><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(x, rows, dp.n, dp.ku, dp.kv, nks, nmt,
                                                                                apack, sc, rpr, rscale ? 1 : 0);
    count_launch();
    LAG_LAUNCH_CHECK();
    gemm_launch(dp, apack, dp.tc_b, rows, y, dp.n, dp.ku, dp.kv, sc, rpr, dp.tc_err, s);
  }
}

void dst_apply_tc_f2d(const DstPlan &dp, const float *y, double *z, int rows, int rpr, const KrylovScalars *sc,
                      cudaStream_t s, bool rscale) {
  if (rows <= 0) return;
  uint8_t *apack = dp.tc_scratch;
  float *eo = reinterpret_cast<float *>(apack + 2 * (size_t)div_up(rows, TM) * dp.kpad_u * 2 * A_TILE);
  const int nks = dp.kpad_u, nmt = div_up(rows, TM);
  {
    ProfScope prof(KC_DSTTC_INV, s);
    const long long threads = (long long)nmt * TM * nks * (TK / 8);
    pack_a_inv_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(y, rows, dp.n, dp.ku, dp.kv, nks, nmt, apack,
                                                                         sc, rpr);
    count_launch();
    LAG_LAUNCH_CHECK();
    gemm_launch(dp, apack, dp.tc_b + 2 * dp.tc_bmat_bytes, rows, eo, 2 * dp.ku, dp.ku, dp.ku, sc, rpr, dp.tc_err, s);
    butterfly_kernel<<<rows, 256, 0, s>>>(eo, z, rows, dp.n, dp.ku, dp.kv, sc, rpr, rscale ? 1 : 0);
    count_launch();
    LAG_LAUNCH_CHECK();
  }
}

void dst_apply_tc_f2d_beta(const DstPlan &dp, const float *y, double *z, int nrhs, int rpr, const double *r,
                           const double *q, int flexible, KrylovScalars *sc, const Reduce &red, cudaStream_t s) {
  const int rows = nrhs * rpr;
  if (rows <= 0) return;
  uint8_t *apack = dp.tc_scratch;
  float *eo = reinterpret_cast<float *>(apack + 2 * (size_t)div_up(rows, TM) * dp.kpad_u * 2 * A_TILE);
  const int nks = dp.kpad_u, nmt = div_up(rows, TM);
  ProfScope prof(KC_DSTTC_INV, s);
  const long long threads = (long long)nmt * TM * nks * (TK / 8);
  pack_a_inv_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(y, rows, dp.n, dp.ku, dp.kv, nks, nmt, apack, sc,
                                                                       rpr);
  count_launch();
  LAG_LAUNCH_CHECK();
  gemm_launch(dp, apack, dp.tc_b + 2 * dp.tc_bmat_bytes, rows, eo, 2 * dp.ku, dp.ku, dp.ku, sc, rpr, dp.tc_err, s);
  // rows per right-hand side over at most min(1216, the reduction's block capacity) blocks
  int blocks = std::min(std::min(rpr, 1216), red.nblk);
  if (blocks < 1) blocks = 1;
  dim3 g(blocks, nrhs);
  butterfly_beta_kernel<<<g, 256, 0, s>>>(eo, z, r, q, dp.n, dp.ku, dp.kv, rpr, flexible, sc, red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void spectrum_permute(const float *in, float *out, int rows, int n, int ku, bool to_perm, cudaStream_t s) {
  const long long t = (long long)rows * n;
  permute_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(in, out, rows, n, ku, to_perm ? 1 : 0);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void spectrum_unpermute_widen(const float *in, double *out, int rows, int n, int ku, cudaStream_t s) {
  const long long t = (long long)rows * n;
  unpermute_widen_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(in, out, rows, n, ku);
  count_launch();
  LAG_LAUNCH_CHECK();
}


// ============================================================================ exact-slice FP64 DST
// The float64 path's transform on the same tensor cores, without rounding anything beyond what a
// float64 GEMM rounds (the Ozaki splitting idea: exact products of short slices, summed in float64).
//   * Every folded input row is scaled by a power of two 2^-e_r with |row| < 2^e_r and cut into
//     NS slices of NB bits of its fixed-point expansion: u = 2^e_r sum_i q_i 2^(-NB i) up to a
//     truncation below 2^(e_r - NS NB) (54 or 56 bits); the q_i are integers |q_i| < 2^NB, exact
//     in bf16 (8-bit significand).  S is sliced the same way with one scale 2^e_B.
//   * A pair (i, j) gives G_ij = sum_k q_i p_j: integers of magnitude < (2^NB - 1)^2 K, exactly
//     summed by the FP32 accumulator while the total stays below 2^24.  Pairs of the same weight
//     i + j share one accumulator in groups of at most floor(2^24 / ((2^NB - 1)^2 K)) (at most 4).
//   * Pairs with i + j <= NS + 1 are kept (the dropped ones weigh < 2^-54 of the row scale), and
//     the epilogue adds the groups as int64 fixed-point numbers (units of 2^-38 of the pre-scaled
//     domain, see oz_fix) and rounds once to float64, y = 2^(e_r + e_B - 2 NB) 2^-FIX I, straight
//     into the float64 output (natural mode order, as the SIMT kernel writes it).  Groups are
//     scheduled in an order that keeps the tensor pipe busy (see oz_schedule).
//   * Slice width: 7 bits (8 slices, 36 pairs) while one pair's exact sum fits the FP32
//     accumulator (127^2 K <= 2^24: K <= 1024), else 6 bits (9 slices, 45 pairs).  The GEMM streams
//     one A and one B slice tile per pair and K step, so fewer pairs mean proportionally fewer
//     operand bytes into each SM, the limit of this kernel.
//   * 8-bit slices (7 balanced digits in [-128, 128] of a 55-bit expansion, 28 pairs; the default
//     up to K = 1024): bf16 holds every such digit exactly and one pair's sum over K <= 1024 stays
//     within 128^2 1024 = 2^24, exact in FP32, so the groups are those of the 7-bit format with
//     22 % fewer products and operand bytes.  (Plain 8-bit digits, up to 255, would need the exact
//     pairs cut into K chunks of 256: 65 accumulator groups per tile instead of 20, and the epilogue
//     then holds the MMA issuer back; the schedule still supports such chunks.)
constexpr int OZ_SMAX = 9;  // slices per operand at most (storage bound)
struct OzFmt {
  int nb, ns;  // bits per slice, slices per operand
};
static OzFmt oz_format(int kpad) {
  const char *v = std::getenv("LAGWAVE_OZ_BITS");  // "7": the 7-bit / 6-bit formats only
  if (kpad <= 1024 && !(v != nullptr && v[0] == '7')) return OzFmt{8, 7};
  return (127LL * 127LL * kpad <= (1LL << 24)) ? OzFmt{7, 8} : OzFmt{6, 9};
}
constexpr int OZ_TN = 128;                 // output columns per tile
constexpr int OZ_BT = OZ_TN * TK * 2;      // B stage tile, 16 KB
constexpr int OZ_KT = 2;                   // 64-wide K tiles per pipeline stage
constexpr int OZ_STAGE = OZ_KT * (A_TILE + OZ_BT);  // 64 KB: [A k tiles][B k tiles]
constexpr int OZ_NST = 3;                  // pipeline stages
constexpr int OZ_NACC = 4;                 // tensor-memory accumulators of 128 columns
constexpr int OZ_SMEM = OZ_NST * OZ_STAGE + 1024 + 256;
// the tile kernel's stages: one K tile of A and of up to two B slices (48 KB), four of them
constexpr int OZT_STAGE = A_TILE + 2 * OZ_BT;
constexpr int OZT_NST = 4;
constexpr int OZT_SMEM = OZT_NST * OZT_STAGE + 1024 + 256;
constexpr int OZ_EXP_NAN = 0x7fffffff;     // row exponent marking a non-finite row
// pairs of weight i + j >= tail share one accumulator with FP32 rounding: together they weigh
// < 2^-(NB (tail - 2)) of the leading products (2^-36 at tail = 8 with 6-bit slices, 2^-42 with
// 7-bit ones, 2^-40 at tail = 7 with 8-bit ones), so that the roundings of the K / 16 accumulating
// MMAs (directed, not random, in the tensor cores' adder: they add up linearly) stay near 2^-50 of
// the row scale or below, under the float64 rounding of the product itself; lighter weights are
// exact.  6-bit slices: tail = 8 up to K = 1024 and one weight later per doubling of K (the
// rounding grows with K); 7-bit slices (K <= 1024): tail = 8 as well (a tail from weight 7, 2^-35,
// measured 1.3e-14 relative row error at K = 1024 against 1e-15 for a float64 GEMM); 8-bit slices
// (K <= 1024): tail = 7.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16_n128(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(OZ_IDESC), "r"(accumulate)
      : "memory");
}

// The schedule of one output tile: a sequence of units (one slice pair over a range of K tiles),
// cut into groups that each fill one tensor-memory accumulator.
constexpr int OZ_MAXU = 128;
struct OzSched {
  int nunits, ngroups, npairs;
  int8_t si[OZ_MAXU], sj[OZ_MAXU];            // slice indices (1-based) of each unit
  uint8_t k0[OZ_MAXU], k1[OZ_MAXU];           // the unit's K tiles [k0, k1)
  int8_t first[OZ_MAXU], last[OZ_MAXU];       // group start / end flags
  int8_t gsh[OZ_MAXU];  // per group: s >= 0 if its sum is an exact integer G with value G 2^-(FIX - s)
                        // (the int64 epilogue adds G << s), -1 for a rounded group (rn(v 2^FIX))
  uint8_t ug[OZ_MAXU];  // group of each unit
  // fused schedules (tile kernel): a second B slice of a unit sharing A slice si (0: none), and
  // split units whose two products fill two consecutive groups (else they share one accumulator)
  int8_t sj2[OZ_MAXU], split[OZ_MAXU];
  int nstage;  // pipeline stages of one tile (OZ_KT K tiles per stage; one for units of two B slices)
};

// The epilogue's accumulator: a signed fixed-point integer in units of 2^-FIX of the pre-scaled
// domain (where weight-2 products have unit 1), in int64.  An exact group of weight w holds
// G 2^-(NB (w - 2)) with G an integer below 2^24: F2I of v 2^(NB (w - 2)) is exact and G << s,
// s = FIX - NB (w - 2) >= 0, places it.  A tail chunk (FP32-rounded, or an exact group too light for
// a non-negative s) is added as rn(v 2^FIX), below 2^31: a rounding at 2^-(FIX+1), under the
// float64 rounding of the product.  FIX = 38: the leading group is at most 2^24 for every format,
// the sum below 2^62.1, and the lightest exact weight keeps s >= 0 (8-bit slices: weight 6, s = 6).
// One I2F and one
// DMUL per output at the end; the per-group work is a float multiply, a conversion and integer adds
// instead of one DFMA on the narrow FP64 pipe.
__host__ __device__ constexpr int oz_fix(int) { return 38; }
// width of the fixed-point expansion of an operand (55 bits for the balanced 8-bit digits, whose top
// digit must stay <= 128), and the exponent shift of its slices: v = 2^(e - se) sum_i q_i 2^-(NB (i-1))
__host__ __device__ constexpr int oz_bits(int nb, int ns) { return nb == 8 ? 55 : nb * ns; }
__host__ __device__ constexpr int oz_se(int nb, int ns) { return oz_bits(nb, ns) - nb * (ns - 1); }

// The epilogue's float64 result RN(v) 2^kx of an int64 sum v (|v| < 2^63), built with integer
// operations: the FP64 pipe of this part runs at 1/64 of the FP32 rate, and an int64 -> float64
// conversion plus two power-of-two scalings per output kept the GEMM's epilogue busy for longer
// than its last group's MMAs.  One rounding, to nearest even, as (double) v rounds.  Only for rows
// whose every result stays in the normal range (oz_fast_row); the others (subnormal or overflowing
// results, non-finite rows) take the float64 expression scale * (unit * (double) v), so every
// output equals that expression's.
__device__ __forceinline__ bool oz_fast_row(int e, int kx) {
  return e != OZ_EXP_NAN && kx + 1023 >= 1 && kx + 64 + 1023 <= 2046;
}
__device__ __forceinline__ double oz_to_f64(long long v, int kx) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long u = sgn ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)u);
  const unsigned long long m = u << (lz & 63);  // leading one at bit 63 (u = 0: m = 0)
  const unsigned long long rem = m & 0x7ffull;
  unsigned long long r = m >> 11;              // 53 bits, the leading one at bit 52
  r += (rem > 0x400ull || (rem == 0x400ull && (r & 1ull))) ? 1ull : 0ull;  // to nearest even
  // exponent field one below the biased exponent, plus r with its leading one: a carry of the
  // rounding into bit 53 raises the exponent by one and leaves a zero fraction
  const unsigned long long ef = (unsigned long long)(63 - lz + kx + 1022) << 52;
  return u == 0 ? 0.0 : __longlong_as_double((long long)(sgn | (ef + r)));
}

// One epilogue thread's outputs of a tile row: the float64 values of its int64 sums (ncols of them,
// ystride doubles apart from yp).
template <bool FAST>
__device__ __forceinline__ void oz_store_row(const long long (&acci)[64], int ncols, int kx, double scale, double unit,
                                             double *yp, int ystride) {
#pragma unroll
  for (int q = 0; q < 64; ++q)
    if (q < ncols) yp[ystride * q] = FAST ? oz_to_f64(acci[q], kx) : scale * (unit * __ll2double_rn(acci[q]));
}
// the same for a row: the integer conversion where every result of the row is a normal float64
__device__ __forceinline__ void oz_store(const long long (&acci)[64], int ncols, int e, int kx, double scale,
                                         double unit, double *yp, int ystride) {
  if (oz_fast_row(e, kx)) oz_store_row<true>(acci, ncols, kx, scale, unit, yp, ystride);
  else oz_store_row<false>(acci, ncols, kx, scale, unit, yp, ystride);
}

// |v| < 2^e: NBITS-bit fixed-point expansion of |v| 2^-e, truncated (integer arithmetic on the bits)
template <int NBITS>
__device__ __forceinline__ unsigned long long oz_fixed(double v, int e) {
  static_assert(NBITS >= 53 && NBITS <= 63, "fixed-point width");
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  const int E = (int)(bits >> 52);
  const unsigned long long M = (bits & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  const int s = (E ? E : 1) - 1075 + NBITS - e;  // |v| = M 2^((E ? E : 1) - 1075)
  if (s >= 0) return M << s;                      // s <= NBITS - 52 since |v| < 2^e
  return (s <= -64) ? 0ull : (M >> (-s));
}
// slice i (1-based) of an NB*NS-bit fixed-point value, pre-scaled by 2^-(NB (i - 1)) and signed, as
// a float whose upper half is the bf16 operand: the integer 0 <= q < 2^NB becomes a float by the
// 2^23 magic-number trick, and one FMA scales it exactly (q has at most 8 significant bits, so the
// low half of the float is zero and its upper half is q 2^-(NB (i - 1)) in bf16; 0 stays +0).
// A product of slices i and j then carries 2^-(NB (i + j - 2)) already, so products of different
// weights can share an accumulator.
// 8-bit slices are balanced digits in [-128, 128] (the 7-bit and 6-bit ones are plain digits): the
// 55-bit value T (below 2^55) plus 128 in each of its six lower byte positions has bytes b_i with
// T = (b_1) 256^6 + sum_{i >= 2} (b_i - 128) 256^(7 - i), b_1 <= 128; every digit magnitude is at
// most 128 = 2^7, so one pair's sum over K <= 1024 stays within 2^24, exact in FP32.
template <int NB, int NS>
__device__ __forceinline__ float oz_slice_f(unsigned long long T, int i, bool neg) {
  static_assert(NB <= 8, "bf16 holds 8 significant bits");
  const float c = __uint_as_float((uint32_t)(127 - NB * (i - 1)) << 23);  // 2^-(NB (i - 1))
  const float cs = neg ? -c : c;
  if constexpr (NB == 8) {
    static_assert(NS == 7, "balanced 8-bit digits of a 55-bit value");
    const unsigned long long Tb = T + 0x0000808080808080ull;
    const uint32_t raw = (uint32_t)(Tb >> (8 * (NS - i))) & (i == 1 ? 0x1ffu : 0xffu);
    const float off = (i == 1) ? 8388608.0f : 8388736.0f;  // 2^23, or 2^23 + 128 for the lower digits
    return fmaf(__uint_as_float(0x4B000000u | raw), cs, -off * cs);
  } else {
    const uint32_t q = (uint32_t)(T >> (NB * NS - NB * i)) & ((1u << NB) - 1u);
    return fmaf(__uint_as_float(0x4B000000u | q), cs, -8388608.0f * cs);
  }
}
__device__ __forceinline__ uint16_t oz_bf16_of(float f) { return (uint16_t)(__float_as_uint(f) >> 16); }
// two slice values as one 32-bit word of bf16 operands (f0 at the lower address)
__device__ __forceinline__ uint32_t oz_pack2(float f0, float f1) {
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// B slices, once per plan: [mat 0, mat 1][slice][n tile][k stage][TN x TK].  Mat w is the row-major
// matrix m_w [K_w][ld_w] (contraction index k, output column n < N_w); zero beyond it.  Forward
// transforms: m0 = su (even output modes), m1 = sv (odd ones); DCT-II inverse: m0 = ie (even input
// modes), m1 = io (odd ones), both with ceil(n/2) output columns.
template <int NB, int NS>
__global__ void oz_pack_b_kernel(const double *m0, int k0n, int n0n, int ld0, const double *m1, int k1n, int n1n,
                                 int ld1, int nks, int nnt, int eB, uint8_t *out, size_t slice_bytes) {
  const int which = blockIdx.z;
  const int n = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnt * OZ_TN || k >= nks * TK) return;
  double v = 0.0;
  if (which == 0) { if (n < n0n && k < k0n) v = m0[(size_t)k * ld0 + n]; }
  else if (n < n1n && k < k1n) v = m1[(size_t)k * ld1 + n];
  const unsigned long long T = oz_fixed<oz_bits(NB, NS)>(v, eB);
  const size_t tile = (size_t)(n / OZ_TN) * nks + (k / TK);
  const uint32_t off = swz(n % OZ_TN, k % TK);
  for (int i = 1; i <= NS; ++i) {
    uint8_t *base = out + ((size_t)which * NS + (i - 1)) * slice_bytes + tile * OZ_BT;
    *reinterpret_cast<uint16_t *>(base + off) = oz_bf16_of(oz_slice_f<NB, NS>(T, i, v < 0.0));
  }
}

// A slices per apply: one CTA of OZ_PACK_THREADS per row, both parities.  Pass 1 stages the row in
// shared memory and takes the row maximum of |input|; pass 2 forms each group of 8 consecutive
// folded values u_j = x_j + x_{n-1-j}, v_j = x_j - x_{n-1-j} as exact sums of the inputs' signed
// fixed-point expansions (at the row exponent one above the largest input, so that the sums keep
// below 2^NBITS), cuts them into slices from the bits and stores them 16 bytes at a time: integer
// operations only (no float64 rounding of the fold, nothing on the narrow FP64 pipe).
// Layout [parity][slice][m tile][k stage][TM x TK]; erow[parity][row] = e_r with |values| < 2^e_r.
constexpr int OZ_PACK_THREADS = 128;  // 62 registers: 128-thread CTAs keep every row of a shot resident at once
constexpr int OZ_PACK_MAXK = 4224;  // ceil(n / 2) bound of the exact-slice path (K pad <= 4224)
// the staged row's index j at j + j / 8: a thread's 8 consecutive values (or the mirrored ones)
// then sit 9 doubles from its neighbour's, so a half-warp's 8-byte reads hit every bank once
// (unpadded, lanes 64 bytes apart fell on two banks: 16-way conflicts)
#define OZ_PAD(j) ((j) + ((j) >> 3))
static size_t oz_pack_smem(int nks) { return (size_t)(2 * nks * TK + (2 * nks * TK) / 8 + 8) * sizeof(double); }
// gather (DCT-II inverse): u = the even entries x[2j], v = the odd ones x[2j+1] instead of the fold.
template <int NB, int NS>
__global__ void __launch_bounds__(OZ_PACK_THREADS) oz_pack_a_kernel(const double *__restrict__ x, int rows, int n,
                                                                    int ku, int kv, int nks, int nmt,
                                                                    uint8_t *__restrict__ out, size_t slice_bytes,
                                                                    int *__restrict__ erow,
                                                                    const KrylovScalars *__restrict__ sc, int rpr,
                                                                    int gather) {
  extern __shared__ double xs[];  // the row's n inputs (n <= 2 nks TK) at OZ_PAD(j)
  const int row = blockIdx.x;
  // rows of finished right-hand sides keep whatever slices they had: the GEMM may still cover them
  // in a tile shared with running rows, but nothing reads those rows' outputs any more (their
  // values stay finite: slices are bounded integers)
  if (row < rows && sc != nullptr && sc[row / rpr].state != ST_RUN) return;
  // the padding rows of the last tile pack as zeros
  const bool live = row < rows;
  const double *xr = x + (size_t)(row < rows ? row : 0) * n;
  const bool odd_n = (n & 1) != 0;
  const int kp = nks * TK;
  // pass 1: stage the row and take the largest |input| (per parity for the gathered DCT-II input) as
  // the largest bit pattern with the sign cleared (the same order for non-negative doubles; NaN and
  // Inf patterns compare above every finite one)
  // (the loads of a batch of 16 per thread all issue before any is used: a whole 2048-long row is
  // in flight at once)
  unsigned long long b0 = 0, b1 = 0;
  constexpr int PB = 16;
  for (int jb = 0; jb < n; jb += PB * blockDim.x) {
    double vb[PB];
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int j = jb + u * blockDim.x + threadIdx.x;
      vb[u] = (live && j < n) ? __ldg(xr + j) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int j = jb + u * blockDim.x + threadIdx.x;
      if (j < n) {
        xs[OZ_PAD(j)] = vb[u];
        const unsigned long long m = (unsigned long long)__double_as_longlong(vb[u]) & 0x7fffffffffffffffull;
        if (gather && (j & 1)) b1 = max(b1, m);
        else b0 = max(b0, m);
      }
    }
  }
  __shared__ unsigned long long red[2][OZ_PACK_THREADS / 32];
  __shared__ int esh[2];
  for (int o = 16; o > 0; o >>= 1) {
    b0 = max(b0, __shfl_xor_sync(0xffffffffu, b0, o));
    b1 = max(b1, __shfl_xor_sync(0xffffffffu, b1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = b0;
    red[1][threadIdx.x >> 5] = b1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int e[2];
    for (int par = 0; par < 2; ++par) {
      unsigned long long m = 0;
      for (int w = 0; w < OZ_PACK_THREADS / 32; ++w) m = max(m, red[gather ? par : 0][w]);
      const int E = (int)(m >> 52);
      // |inputs| <= m < 2^(E - 1022) for normal m, < 2^-1022 for subnormal m; 0 for a zero row.
      // The fold's sums and differences of two inputs stay below 2^(that + 1).
      e[par] = (E == 0x7ff) ? OZ_EXP_NAN : (m == 0 ? 0 : (E == 0 ? -1022 : E - 1022) + (gather ? 0 : 1));
    }
    // a non-finite value anywhere in the row makes every output of the row non-finite, as in a
    // float64 product (the middle element of an odd-length row reaches one parity only, yet its
    // zero coefficient in the other parity's modes still gives inf x 0 = NaN there)
    if (e[0] == OZ_EXP_NAN || e[1] == OZ_EXP_NAN) e[0] = e[1] = OZ_EXP_NAN;
    for (int par = 0; par < 2; ++par) {
      esh[par] = e[par];
      if (row < rows) erow[par * (nmt * TM) + row] = e[par];
    }
  }
  __syncthreads();
  const int mt = row / TM, r = row % TM;
  const bool bad = esh[0] == OZ_EXP_NAN;
  const int e0 = bad ? 0 : esh[0], e1 = bad ? 0 : esh[1];
  // signed NBITS-bit fixed-point value of an input at exponent e (|input| < 2^(e-1) for the fold)
  auto sfix = [&](double v, int e) -> long long {
    const long long t = (long long)oz_fixed<oz_bits(NB, NS)>(v, e);
    return __double_as_longlong(v) < 0 ? -t : t;
  };
  // pass 2: one 8-value chunk of both parities per thread and step.  The fold's sums and
  // differences are exact integer sums of the inputs' expansions (no float64 rounding, no FP64 pipe)
  for (int ch = threadIdx.x; ch < kp / 8; ch += blockDim.x) {
    const int k0 = ch * 8, ks = k0 / TK, kk = k0 % TK;
    long long S[2][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = k0 + q;
      long long u = 0, w = 0;
      if (!bad) {
        if (gather) {
          if (j < ku) u = sfix(xs[OZ_PAD(2 * j)], e0);
          if (j < kv) w = sfix(xs[OZ_PAD(2 * j + 1)], e1);
        } else if (j < kv) {
          const long long a1 = sfix(xs[OZ_PAD(j)], e0), a2 = sfix(xs[OZ_PAD(n - 1 - j)], e0);
          u = a1 + a2;
          w = a1 - a2;
        } else if (odd_n && j == ku - 1) {
          u = sfix(xs[OZ_PAD(j)], e0);  // middle element of an odd-length row
        }
      }
      S[0][q] = u;
      S[1][q] = w;
    }
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      unsigned long long T[8];
      uint32_t negm = 0;
  #pragma unroll
      for (int q = 0; q < 8; ++q) {
        const long long v = S[par][q];
        T[q] = (unsigned long long)(v < 0 ? -v : v);
        negm |= (v < 0 ? 1u : 0u) << q;
      }
      const uint32_t off = swz(r, kk);
      uint8_t *tile0 = out + (size_t)par * NS * slice_bytes + ((size_t)mt * nks + ks) * A_TILE + off;
      if constexpr (NB == 8) {
        // balanced digits straight from the bytes of T + 128 (256^0 + ... + 256^5), split into two
        // 32-bit words: one byte permute builds 2^23 + byte as a float, one subtraction and one
        // power-of-two multiply give the signed, pre-scaled digit (the same values as oz_slice_f)
        uint32_t th[8], tl[8];
  #pragma unroll
        for (int q = 0; q < 8; ++q) {
          const unsigned long long Tb = T[q] + 0x0000808080808080ull;
          tl[q] = (uint32_t)Tb;
          th[q] = (uint32_t)(Tb >> 32);
        }
  #pragma unroll
        for (int i = 1; i <= NS; ++i) {
          const uint32_t cbits = (uint32_t)(127 - 8 * (i - 1)) << 23;  // 2^-(8 (i - 1))
          const float offv = (i == 1) ? 8388608.0f : 8388736.0f;
          uint32_t hw[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            float d[2];
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int v = 2 * q + h;
              uint32_t fb;
              if (i == 1) fb = 0x4B000000u | ((th[v] >> 16) & 0x1ffu);
              else if (i <= 3) fb = __byte_perm(th[v], 0x4B00u, 0x5440u | (uint32_t)(3 - i));
              else fb = __byte_perm(tl[v], 0x4B00u, 0x5440u | (uint32_t)(7 - i));
              const float cq = __uint_as_float(cbits | (((negm >> v) & 1u) << 31));
              d[h] = (__uint_as_float(fb) - offv) * cq;
            }
            hw[q] = oz_pack2(d[0], d[1]);
          }
          *reinterpret_cast<uint4 *>(tile0 + (size_t)(i - 1) * slice_bytes) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        }
      } else {
  #pragma unroll
        for (int i = 1; i <= NS; ++i) {
          uint32_t hw[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q)
            hw[q] = oz_pack2(oz_slice_f<NB, NS>(T[2 * q], i, (negm >> (2 * q)) & 1u),
                             oz_slice_f<NB, NS>(T[2 * q + 1], i, (negm >> (2 * q + 1)) & 1u));
          *reinterpret_cast<uint4 *>(tile0 + (size_t)(i - 1) * slice_bytes) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        }
      }
    }
  }
}

// Persistent warp-specialised GEMM over (parity, m tile, n tile) tiles and, per tile, the fused
// pair schedule: warp 0 streams the stages of each unit (two K tiles of A_i and B_j, or one K tile
// of A_i, B_j and B_j2), warp 1 issues the MMAs of a group into one of four tensor-memory
// accumulators, warps 2-9 add finished groups into int64 sums held in registers (warp w: rows
// 32 (w % 4).., columns 64 ((w - 2) / 4)..) and store the tile once at its end.
template <int NB, int NS>
__global__ void __launch_bounds__(320, 1) oz_gemm_kernel(const uint8_t *__restrict__ apack, size_t a_slice_bytes,
                                                         const uint8_t *__restrict__ bpack, size_t b_slice_bytes,
                                                         const int *__restrict__ erow, int eB, int nks, int nmt,
                                                         int nnt, int rows, double *__restrict__ y, int ld, int ku,
                                                         int kv, OzSched sch, const KrylovScalars *__restrict__ sc,
                                                         int rpr, int *__restrict__ err, int inv) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  const uint32_t bars = base + OZT_NST * OZT_STAGE;
  const uint32_t full0 = bars, empty0 = bars + 8 * OZT_NST, tfull0 = bars + 16 * OZT_NST, tempty0 = tfull0 + 8 * OZ_NACC;
  volatile uint32_t *holder =
      reinterpret_cast<volatile uint32_t *>(gbase + OZT_NST * OZT_STAGE + 16 * OZT_NST + 16 * OZ_NACC + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + OZT_NST * OZT_STAGE + 16 * OZT_NST + 16 * OZ_NACC + 16);
  // the tile whose int64 sums the epilogue left in the stage buffers for the whole CTA to store (-1: none)
  volatile int *tail_tile = reinterpret_cast<volatile int *>(gbase + OZT_NST * OZT_STAGE + 16 * OZT_NST + 16 * OZ_NACC + 24);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = 2 * nmt * nnt;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)holder)),
                 "r"(OZ_NACC * OZ_TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < OZT_NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < OZ_NACC; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 8);  // one arrive per epilogue warp
    }
    *abort_flag = 0;
    *tail_tile = -1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;

  auto decode = [&](int t, int &par, int &mt, int &nt) {
    nt = t % nnt;
    mt = (t / nnt) % nmt;
    par = t / (nnt * nmt);
  };
  auto wanted = [&](int par, int mt, int nt) -> bool {
    if (nt * OZ_TN >= ((par && !inv) ? kv : ku)) return false;
    if (mt * TM >= rows) return false;  // the padding m-tile of an odd count (A slices come in pairs)
    if (sc == nullptr) return true;
    const int m0 = mt * TM;
    const int r0 = m0 / rpr, r1 = (min(m0 + TM, rows) - 1) / rpr;
    for (int r = r0; r <= r1; ++r)
      if (sc[r].state == ST_RUN) return true;
    return false;
  };

  if (warp == 0) {
    if (lane == 0) {  // producer: per stage one K tile of A_i and of its one or two B_j
      int s = 0, it = 0;
      uint32_t ph = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int par, mt, nt;
        decode(t, par, mt, nt);
        if (!wanted(par, mt, nt)) continue;
        for (int pr = 0; pr < sch.nunits && !*abort_flag; ++pr) {
          const uint8_t *at = apack + ((size_t)par * NS + (sch.si[pr] - 1)) * a_slice_bytes + (size_t)mt * nks * A_TILE;
          const uint8_t *bt = bpack + ((size_t)par * NS + (sch.sj[pr] - 1)) * b_slice_bytes + (size_t)nt * nks * OZ_BT;
          const bool two = sch.sj2[pr] > 0;
          const uint8_t *bt2 =
              bpack + ((size_t)par * NS + (max((int)sch.sj2[pr], 1) - 1)) * b_slice_bytes + (size_t)nt * nks * OZ_BT;
          for (int kk = sch.k0[pr]; kk < sch.k1[pr]; ++kk) {
            if (it >= OZT_NST && !mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
              atomicExch(err, 11);
              *abort_flag = 1;
              break;
            }
            const uint32_t st = base + s * OZT_STAGE;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, (uint32_t)(A_TILE + (two ? 2 : 1) * OZ_BT));
            bulk_g2s(st, at + (size_t)kk * A_TILE, A_TILE, fb);
            bulk_g2s(st + A_TILE, bt + (size_t)kk * OZ_BT, OZ_BT, fb);
            if (two) bulk_g2s(st + A_TILE + OZ_BT, bt2 + (size_t)kk * OZ_BT, OZ_BT, fb);
            ++it;
            if (++s == OZT_NST) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      // stage ring position and phase kept incrementally; shared-memory descriptors as one OR of
      // the constant upper bits with the stage's 16-byte address (the issuer is a single thread:
      // its per-stage arithmetic is time the tensor pipe may sit idle)
      constexpr uint64_t DHI = ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61) | (1ull << 16);
      constexpr uint32_t B1 = A_TILE >> 4, B2 = (A_TILE + OZ_BT) >> 4;
      int s = 0, gc = 0;
      uint32_t ph = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int par, mt, nt;
        decode(t, par, mt, nt);
        if (!wanted(par, mt, nt)) continue;
        uint32_t d = 0;
        for (int pr = 0; pr < sch.nunits && !*abort_flag; ++pr) {
          const bool split = sch.split[pr] != 0, first = sch.first[pr] != 0, two = sch.sj2[pr] > 0;
          if (first) {
            bool ok = true;
            for (int q = 0; q < (split ? 2 : 1); ++q) {  // a split unit fills two accumulators
              const int acc = (gc + q) % OZ_NACC, ause = (gc + q) / OZ_NACC;
              if (gc + q >= OZ_NACC && !mbar_wait(tempty0 + 8 * acc, (ause - 1) & 1)) ok = false;
            }
            if (!ok) {
              atomicExch(err, 14);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            d = tmem + (uint32_t)((gc % OZ_NACC) * OZ_TN);
          }
          // the second B slice's products go to the same accumulator, or (split) the next group's;
          // a fresh accumulator takes its first product without accumulating (the group's first K
          // tile, for the first product and for the second of a split unit)
          const uint32_t d2 = split ? tmem + (uint32_t)(((gc + 1) % OZ_NACC) * OZ_TN) : d;
          const int kb = sch.k0[pr], ke = sch.k1[pr];
          for (int kk = kb; kk < ke; ++kk) {
            if (!mbar_wait(full0 + 8 * s, ph)) {
              atomicExch(err, 12);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = (base + s * OZT_STAGE) >> 4;
            const uint32_t f1 = (first && kk == kb) ? 0u : 1u;
#pragma unroll
            for (int sub = 0; sub < TK / 16; ++sub)
              mma_bf16_n128(d, DHI | (sa + 2 * sub), DHI | (sa + B1 + 2 * sub), sub == 0 ? f1 : 1u);
            if (two) {
              const uint32_t f2 = split ? f1 : 1u;
#pragma unroll
              for (int sub = 0; sub < TK / 16; ++sub)
                mma_bf16_n128(d2, DHI | (sa + 2 * sub), DHI | (sa + B2 + 2 * sub), sub == 0 ? f2 : 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                         : "memory");
            if (++s == OZT_NST) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (sch.last[pr]) {
            for (int q = 0; q < (split ? 2 : 1); ++q) {
              asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                               tfull0 + 8 * ((gc + q) % OZ_NACC))
                           : "memory");
            }
            gc += split ? 2 : 1;
          }
        }
      }
    }
  } else {  // epilogue warps 2..9
    const int lg = warp & 3, h = (warp - 2) >> 2;
    int gc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int par, mt, nt;
      decode(t, par, mt, nt);
      if (!wanted(par, mt, nt)) continue;
      const int row = mt * TM + lg * 32 + lane;
      const bool rok = row < rows;
      const int e = rok ? erow[par * (nmt * TM) + row] : 0;
      long long acci[64];
#pragma unroll
      for (int q = 0; q < 64; ++q) acci[q] = 0;
      bool stop = false;
      for (int g = 0; g < sch.ngroups; ++g) {
        const int acc = gc % OZ_NACC, ause = gc / OZ_NACC;
        const bool ok = mbar_wait(tfull0 + 8 * acc, ause & 1);
        __syncwarp();
        if (!ok) {
          if (lane == 0) atomicExch(err, 13);
          *abort_flag = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int gs = sch.gsh[g];
        // exact: G = v 2^(38 - s) exactly (a power-of-two multiply), then G << s; rounded: rn(v 2^38)
        constexpr int FIX = oz_fix(NB);
        const float up = __uint_as_float((uint32_t)(127 + (gs >= 0 ? FIX - gs : FIX)) << 23);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * OZ_TN + h * 64 + c * 16), v);
          if (gs >= 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rz(v[q] * up) << gs;
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rn(v[q] * up);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * acc) : "memory");
        ++gc;
      }
      if (stop) break;
      if (t + (int)gridDim.x >= ntiles) {
        // the CTA's last tile: once its last group is in, every MMA and every copy of the CTA is
        // complete and the stage buffers are free.  The sums go there ([128 rows][128 columns] int64,
        // column index XOR (row & 7) << 1: the rows' 16-byte writes and the columns' 8-byte reads
        // below meet every bank once per wavefront), and the whole CTA converts and stores them.
        long long *dump = reinterpret_cast<long long *>(gbase);
        const int rl = lg * 32 + lane;
#pragma unroll
        for (int q = 0; q < 64; q += 2)
          *reinterpret_cast<longlong2 *>(dump + rl * OZ_TN + ((h * 64 + q) ^ ((rl & 7) << 1))) =
              make_longlong2(acci[q], acci[q + 1]);
        if (h == 0) reinterpret_cast<int *>(dump + TM * OZ_TN)[rl] = e;  // the rows' exponents after the sums
        if (warp == 2 && lane == 0) *tail_tile = t;
      } else if (rok) {
        // the one float64 rounding of the product: int64 -> double, then exact power-of-two scales
        // (2^-38 first, so that a row near the bottom of the float64 range meets the same
        // subnormal rounding as its float64 product would); built from integer operations where
        // every result of the row is a normal float64
        const double scale = (e == OZ_EXP_NAN) ? __longlong_as_double(0x7ff8000000000000ll)
                                               : ldexp(1.0, e + eB - 2 * oz_se(NB, NS));
        const double unit = 1.0 / (double)(1LL << oz_fix(NB));
        const int kx = e + eB - 2 * oz_se(NB, NS) - oz_fix(NB);
        const int c0 = nt * OZ_TN + h * 64;
        const int ncols = min(64, ((par && !inv) ? kv : ku) - c0);
        // DCT-II inverse: the even / odd mode sums E, O as [par][row][ku]; else the interleaved spectrum
        const size_t o = inv ? ((size_t)par * rows + row) * ku + c0 : (size_t)row * ld + par + 2 * (size_t)c0;
        oz_store(acci, ncols, e, kx, scale, unit, y + o, inv ? 1 : 2);
      }
    }
  }
  // the last tile's store: ten warps, one row at a time (the row's scale and the integer / float64
  // choice uniform over the warp), lanes along the row's columns.  With the sums in registers, the
  // eight epilogue warps converted and stored 64 values each after the last MMA with few registers
  // left; here the conversion runs at the integer pipe's rate (about one value per clock and SM)
  __syncthreads();
  const int tt = *tail_tile;
  if (tt >= 0) {
    int par, mt, nt;
    decode(tt, par, mt, nt);
    const long long *dump = reinterpret_cast<const long long *>(gbase);
    const int c0 = nt * OZ_TN;
    const int ncols = min(OZ_TN, ((par && !inv) ? kv : ku) - c0);
    const int ys = inv ? 1 : 2;
    const int *esh = reinterpret_cast<const int *>(dump + TM * OZ_TN);
    for (int rl = warp; rl < TM; rl += 10) {
      const int row = mt * TM + rl;
      if (row >= rows) break;
      const int e = esh[rl];
      const int kx = e + eB - 2 * oz_se(NB, NS) - oz_fix(NB);
      double *yr = y + (inv ? ((size_t)par * rows + row) * ku + c0 : (size_t)row * ld + par + 2 * (size_t)c0);
      const long long *dr = dump + rl * OZ_TN;
      const int sw = (rl & 7) << 1;
      if (oz_fast_row(e, kx)) {
        // the FP64 pipe's int64 -> float64 conversion (the one rounding, to nearest even), then kx
        // added to the exponent field: exact, as every result of such a row stays normal; the same
        // bits as oz_to_f64, which took the integer pipe about 17 k clocks per tile (14 k here)
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const int col = k4 * 32 + lane;
          const long long d = __double_as_longlong(__ll2double_rn(dr[col ^ sw]));
          if (col < ncols) yr[ys * col] = __longlong_as_double(d == 0 ? 0ll : d + ((long long)kx << 52));
        }
      } else {
        const double scale = (e == OZ_EXP_NAN) ? __longlong_as_double(0x7ff8000000000000ll)
                                               : ldexp(1.0, e + eB - 2 * oz_se(NB, NS));
        const double unit = 1.0 / (double)(1LL << oz_fix(NB));
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const int col = k4 * 32 + lane;
          const long long a = dr[col ^ sw];
          if (col < ncols) yr[ys * col] = scale * (unit * __ll2double_rn(a));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_NACC * OZ_TN) : "memory");
}

// ---------------------------------------------------------------- stream-K variant
// The same GEMM (forward transforms of one right-hand side) with the sequence of (tile, pipeline
// stage) steps of all tiles cut into one equal range per CTA, one CTA per SM, so that every SM gets
// the same work when the tile count is not a multiple of the SM count (a 2048 x 1024 field: 128
// tiles on 152 SMs).  A range that starts or ends inside a group accumulates that part alone; the
// parts of a group are added in int64 (exact for exact groups; a rounded group is rounded once per
// part, each within the group's bound).
// A tile that no one CTA covers whole is finished by the CTA holding its last step (the finaliser).
// A CTA whose range starts inside a tile runs its range rotated: from the next tile boundary to its
// end, then its first steps, so that the finaliser holds its own part in registers when it comes to
// finish the tile.  Every other part (the end of a range, or a range inside one tile) goes to the
// CTA's slot of `part` as int64, column-major, with a flag per epilogue warp set to the launch's
// mark; the finaliser waits (bounded) for the flags of the CTAs before it that touch the tile, adds
// their parts and stores the tile.  CTAs take their range index from a ticket counter as they
// start, so a CTA only waits for CTAs that started before it, and those write their parts before
// they wait for anything: the hand-over cannot deadlock, whatever the order in which the hardware
// places the CTAs or other work shares the GPU.  The last CTA to finish resets the counters and
// advances the epoch, so flags left by an aborted launch never match a later launch's mark.
constexpr int OZ_SK_MAXG = 256;  // CTAs of a stream-K launch at most
struct OzSkArea {
  long long *part;  // [G][TN][TM] int64 partial tiles, one slot per CTA
  int *ctl;         // ticket, finished, epoch (64 ints reserved)
  int *flag;        // [G][8]
};
template <int NB, int NS>
__global__ void __launch_bounds__(320, 1) oz_gemm_sk_kernel(const uint8_t *__restrict__ apack, size_t a_slice_bytes,
                                                            const uint8_t *__restrict__ bpack, size_t b_slice_bytes,
                                                            const int *__restrict__ erow, int eB, int nks, int nmt,
                                                            int nnt, int rows, double *__restrict__ y, int ld, int ku,
                                                            int kv, OzSched sch, const KrylovScalars *__restrict__ sc,
                                                            int *__restrict__ err, OzSkArea ska) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  const uint32_t bars = base + OZ_NST * OZ_STAGE;
  const uint32_t full0 = bars, empty0 = bars + 8 * OZ_NST, tfull0 = bars + 16 * OZ_NST, tempty0 = tfull0 + 8 * OZ_NACC;
  volatile uint32_t *holder =
      reinterpret_cast<volatile uint32_t *>(gbase + OZ_NST * OZ_STAGE + 16 * OZ_NST + 16 * OZ_NACC + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + OZ_NST * OZ_STAGE + 16 * OZ_NST + 16 * OZ_NACC + 16);
  volatile int *shared_ticket = abort_flag + 1;  // [ticket, epoch]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)holder)),
                 "r"(OZ_NACC * OZ_TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < OZ_NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < OZ_NACC; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 8);  // one arrive per epilogue warp
    }
    *abort_flag = 0;
    int t = atomicAdd(ska.ctl, 1);
    if (t < 0 || t >= G) {  // counters not reset: nothing is computed, the solve reports it
      atomicExch(err, 36);
      t = G;
    }
    shared_ticket[0] = t;
    shared_ticket[1] = *reinterpret_cast<volatile int *>(ska.ctl + 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;
  const int d = shared_ticket[0];         // this CTA's range index (order of start)
  const int mark = shared_ticket[1] + 1;  // flag value of this launch
  const bool run = sc == nullptr || sc[0].state == ST_RUN;  // one right-hand side
  const int nmtv = (rows + TM - 1) / TM;
  const int nnt0 = (ku + OZ_TN - 1) / OZ_TN, nnt1 = (kv + OZ_TN - 1) / OZ_TN;
  const int S = sch.nstage;
  const int total = (run && d < G) ? nmtv * (nnt0 + nnt1) * S : 0;
  auto range_b = [&](int c) { return (int)((long long)c * total / G); };
  const int sk_b = range_b(d), sk_e = range_b(d + 1);
  // the tile of the first step; a range starting inside it runs [x0, sk_e) and then [sk_b, x0)
  const int vt0 = sk_b / (S > 0 ? S : 1);
  const int x0 = (sk_b > vt0 * S) ? min(sk_e, (vt0 + 1) * S) : sk_b;
  const bool finaliser = sk_b > vt0 * S && x0 == (vt0 + 1) * S;
  auto tile_of = [&](int v, int &par, int &mt, int &nt) {
    const int n0 = nmtv * nnt0;
    par = v >= n0 ? 1 : 0;
    const int w = v - par * n0, nn = par ? nnt1 : nnt0;
    mt = w / nn;
    nt = w - mt * nn;
  };
  // position of step s0: tile v, unit u and its K tile kk
  auto locate = [&](int s0, int &v, int &u, int &kk) {
    v = s0 / S;
    int rem = s0 - v * S;
    u = 0;
    for (;;) {
      const int nst = (sch.k1[u] - sch.k0[u] + OZ_KT - 1) / OZ_KT;
      if (rem < nst) break;
      rem -= nst;
      ++u;
    }
    kk = sch.k0[u] + rem * OZ_KT;
  };

  if (warp == 0) {
    if (lane == 0) {  // producer
      int it = 0;
      for (int pass = 0; pass < 2 && !*abort_flag; ++pass) {
        const int rb = pass ? sk_b : x0, re = pass ? x0 : sk_e;
        if (rb >= re) continue;
        int v, u, kk, par, mt, nt;
        locate(rb, v, u, kk);
        tile_of(v, par, mt, nt);
        const uint8_t *at = apack + ((size_t)par * NS + (sch.si[u] - 1)) * a_slice_bytes + (size_t)mt * nks * A_TILE;
        const uint8_t *bt = bpack + ((size_t)par * NS + (sch.sj[u] - 1)) * b_slice_bytes + (size_t)nt * nks * OZ_BT;
        for (int s = rb; s < re && !*abort_flag; ++s, ++it) {
          const int kt = min(OZ_KT, sch.k1[u] - kk);
          const int st_i = it % OZ_NST, use = it / OZ_NST;
          if (it >= OZ_NST && !mbar_wait(empty0 + 8 * st_i, (use - 1) & 1)) {
            atomicExch(err, 31);
            *abort_flag = 1;
            break;
          }
          const uint32_t st = base + st_i * OZ_STAGE;
          const uint32_t fb = full0 + 8 * st_i;
          mbar_expect_tx(fb, (uint32_t)(kt * (A_TILE + OZ_BT)));
          bulk_g2s(st, at + (size_t)kk * A_TILE, (uint32_t)(kt * A_TILE), fb);
          bulk_g2s(st + OZ_KT * A_TILE, bt + (size_t)kk * OZ_BT, (uint32_t)(kt * OZ_BT), fb);
          kk += OZ_KT;
          if (kk >= sch.k1[u]) {  // the next unit, or the next tile's first
            if (++u == sch.nunits) {
              u = 0;
              if (s + 1 < re) tile_of(++v, par, mt, nt);
            }
            kk = sch.k0[u];
            at = apack + ((size_t)par * NS + (sch.si[u] - 1)) * a_slice_bytes + (size_t)mt * nks * A_TILE;
            bt = bpack + ((size_t)par * NS + (sch.sj[u] - 1)) * b_slice_bytes + (size_t)nt * nks * OZ_BT;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int it = 0, gc = 0;
      uint32_t dacc = 0;
      for (int pass = 0; pass < 2 && !*abort_flag; ++pass) {
        const int rb = pass ? sk_b : x0, re = pass ? x0 : sk_e;
        if (rb >= re) continue;
        int v, u, kk;
        locate(rb, v, u, kk);
        for (int s = rb; s < re && !*abort_flag; ++s, ++it) {
          const int kt = min(OZ_KT, sch.k1[u] - kk);
          const bool start = s == rb || (kk == sch.k0[u] && sch.first[u]);
          const bool end = s + 1 == re || (kk + OZ_KT >= sch.k1[u] && sch.last[u]);
          if (start) {
            const int acc = gc % OZ_NACC, ause = gc / OZ_NACC;
            if (gc >= OZ_NACC && !mbar_wait(tempty0 + 8 * acc, (ause - 1) & 1)) {
              atomicExch(err, 32);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            dacc = tmem + (uint32_t)(acc * OZ_TN);
          }
          const int st_i = it % OZ_NST, use = it / OZ_NST;
          if (!mbar_wait(full0 + 8 * st_i, use & 1)) {
            atomicExch(err, 33);
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = base + st_i * OZ_STAGE;
          for (int t = 0; t < kt; ++t) {
#pragma unroll
            for (int sub = 0; sub < TK / 16; ++sub) {
              const uint32_t o = sub * 32;
              mma_bf16_n128(dacc, sdesc(st + t * A_TILE + o), sdesc(st + OZ_KT * A_TILE + t * OZ_BT + o),
                            (start && t == 0 && sub == 0) ? 0u : 1u);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           empty0 + 8 * st_i)
                       : "memory");
          if (end) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tfull0 + 8 * (gc % OZ_NACC))
                         : "memory");
            ++gc;
          }
          kk += OZ_KT;
          if (kk >= sch.k1[u]) {
            if (++u == sch.nunits) u = 0;
            kk = sch.k0[u];
          }
        }
      }
    }
  } else {  // epilogue warps 2..9
    const int lg = warp & 3, h = (warp - 2) >> 2, ew = warp - 2;
    // this lane's part of a tile in a slot: row lg*32 + lane, columns h*64 + q (column-major)
    const size_t pofs = (size_t)(h * 64) * TM + lg * 32 + lane;
    int gc = 0;
    bool stop = false;
    long long acci[64];
    for (int pass = 0; pass < 2 && !stop; ++pass) {
      const int rb = pass ? sk_b : x0, re = pass ? x0 : sk_e;
      if (rb >= re) continue;
      int v, u, kk;
      locate(rb, v, u, kk);
      int s = rb;
      while (s < re && !stop) {  // one segment: the steps of one tile in [rb, re)
        const int vt = v, seg_b = s;
#pragma unroll
        for (int q = 0; q < 64; ++q) acci[q] = 0;
        while (s < re && v == vt) {  // one accumulator: a group, or its part in [rb, re)
          const int g = sch.ug[u];
          for (;;) {
            const bool end = s + 1 == re || (kk + OZ_KT >= sch.k1[u] && sch.last[u]);
            ++s;
            kk += OZ_KT;
            if (kk >= sch.k1[u]) {
              if (++u == sch.nunits) {
                u = 0;
                ++v;
              }
              kk = sch.k0[u];
            }
            if (end) break;
          }
          const int acc = gc % OZ_NACC, ause = gc / OZ_NACC;
          const bool ok = mbar_wait(tfull0 + 8 * acc, ause & 1);
          __syncwarp();
          if (!ok) {
            if (lane == 0) atomicExch(err, 34);
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int gs = sch.gsh[g];
          constexpr int FIX = oz_fix(NB);
          const float up = __uint_as_float((uint32_t)(127 + (gs >= 0 ? FIX - gs : FIX)) << 23);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float vv[16];
            tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * OZ_TN + h * 64 + c * 16), vv);
            if (gs >= 0) {
#pragma unroll
              for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rz(vv[q] * up) << gs;
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rn(vv[q] * up);
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * acc) : "memory");
          ++gc;
        }
        if (stop) break;
        const bool whole = seg_b == vt * S && s == (vt + 1) * S;
        if (!whole && !(finaliser && seg_b == sk_b)) {
          // a part finished by a later CTA: to this CTA's slot, then the flag
          long long *pp = ska.part + (size_t)d * TM * OZ_TN + pofs;
#pragma unroll
          for (int q = 0; q < 64; ++q) __stcg(pp + (size_t)q * TM, acci[q]);
          __threadfence();
          __syncwarp();
          if (lane == 0)
            asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(ska.flag + d * 8 + ew), "r"(mark) : "memory");
          continue;
        }
        if (!whole) {
          // finaliser: add the parts of the earlier CTAs whose ranges reach into the tile
          for (int c = d - 1; c >= 0; --c) {
            const int cb = range_b(c), ce = range_b(c + 1);
            if (ce <= vt * S) break;  // this range and the earlier ones end before the tile
            if (cb == ce) continue;
            int got = 1;
            if (lane == 0) {
              long long i = 0;
              for (; i < WAIT_LIMIT; ++i) {
                int fv;
                asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(fv) : "l"(ska.flag + c * 8 + ew) : "memory");
                if (fv == mark) break;
                if (i > 32) __nanosleep(64);
              }
              got = i < WAIT_LIMIT ? 1 : 0;
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            __syncwarp();  // the lanes' loads below come after lane 0's acquire
            if (!got) {
              if (lane == 0) atomicExch(err, 35);
              *abort_flag = 1;
              stop = true;
              break;
            }
            const long long *pp = ska.part + (size_t)c * TM * OZ_TN + pofs;
#pragma unroll
            for (int q = 0; q < 64; ++q) acci[q] += __ldcg(pp + (size_t)q * TM);
            if (cb <= vt * S) break;  // the part holding the tile's first step
          }
          if (stop) break;
        }
        // the tile: one float64 rounding of each int64 sum, then the power-of-two scales
        int par, mt, nt;
        tile_of(vt, par, mt, nt);
        const int row = mt * TM + lg * 32 + lane;
        if (row < rows) {
          const int e = erow[par * (nmt * TM) + row];
          const double scale = (e == OZ_EXP_NAN) ? __longlong_as_double(0x7ff8000000000000ll)
                                                 : ldexp(1.0, e + eB - 2 * oz_se(NB, NS));
          const double unit = 1.0 / (double)(1LL << oz_fix(NB));
          const int kx = e + eB - 2 * oz_se(NB, NS) - oz_fix(NB);
          const int c0 = nt * OZ_TN + h * 64;
          const int ncols = min(64, (par ? kv : ku) - c0);
          const size_t o = (size_t)row * ld + par + 2 * (size_t)c0;
          oz_store(acci, ncols, e, kx, scale, unit, y + o, 2);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_NACC * OZ_TN) : "memory");
  if (tid == 0) {  // the last CTA out resets the ticket and finish counters and advances the epoch
    __threadfence();
    if (atomicAdd(ska.ctl + 1, 1) == G - 1) {
      atomicExch(ska.ctl, 0);
      atomicExch(ska.ctl + 1, 0);
      atomicAdd(ska.ctl + 2, 1);
    }
  }
}

// ---------------------------------------------------------------- two-SM (cta_group::2) variant
// The same exact-slice GEMM with the MMA spread over a cluster of two CTAs on two SMs: the pair
// computes a 256 x 128 tile per (pair, K step), each CTA holding its own 128 rows of A and half of
// the 128 B columns in shared memory; the tensor cores of the pair exchange the B halves.  With the
// tile kernel's fused schedule (a K tile of A_i with one or two B_j per stage) each SM streams
// 16 + 8 or 16 + 16 KB per 4 or 8 MMAs of 128 x 128 x 16 of its own output instead of 16 + 16 or
// 16 + 32 KB (the per-SM operand stream is what bounds the one-CTA kernel).  The MMAs are issued by one thread of
// the even CTA (the leader) into both CTAs' tensor memory; each CTA's epilogue adds its own rows.
// Synchronisation across the pair: both CTAs' operand copies (TMA tensor copies of the pre-swizzled
// slice tiles, verbatim rows of 128 bytes) complete on the leader's "full" barrier, whose expected
// byte count the leader sets for the pair; the leader's commits arrive on both CTAs' "empty" and
// "tfull" barriers (multicast); the odd CTA's epilogue warps arrive on the leader's "tempty".  Every wait is bounded; both CTAs meet at a cluster barrier before
// they free their tensor memory and exit, so neither leaves while the other may still use it.
constexpr int OZ2_BH = (OZ_TN / 2) * TK * 2;            // half a B K tile: 64 columns x 64 K, 8 KB
constexpr int OZ2_ROWB = 2048;                          // bytes per row of the slice buffers' tensor maps
constexpr int OZ2_STAGE = A_TILE + 2 * OZ2_BH;          // 32 KB: one K tile of A and up to two B halves
constexpr int OZ2_NST = 6;                              // pipeline stages
constexpr int OZ2_NACC = 4;                             // accumulators of 128 columns per CTA
constexpr int OZ2_SMEM = OZ2_NST * OZ2_STAGE + 1024 + 512;
// kind::f16, D f32, A / B bf16 K-major, M = 256 (the pair), N = 128
constexpr uint32_t OZ2_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_TN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait with cluster-scope acquire (for barriers that another CTA's threads arrive on)
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (i > 32) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void mma2_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(OZ2_IDESC), "r"(accumulate)
      : "memory");
}
// TMA copy of rows [y, y + box rows) of a 2-D tensor of 128-byte rows into this CTA's shared memory,
// completing on the mbarrier at cluster address `bar` (this CTA's or its pair leader's)
__device__ __forceinline__ void tma_rows2(uint32_t dst, const CUtensorMap *tm, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void commit2_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"((uint16_t)3)
      : "memory");
}

template <int NB, int NS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(320, 1)
    oz_gemm2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const int *__restrict__ erow, int eB, int nks, int nmt, int nnt, int rows,
                    double *__restrict__ y, int ld, int ku, int kv, OzSched sch, const KrylovScalars *__restrict__ sc,
                    int rpr, int *__restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  const uint32_t bars = base + OZ2_NST * OZ2_STAGE;
  const uint32_t full0 = bars, empty0 = bars + 8 * OZ2_NST;
  const uint32_t tfull0 = bars + 16 * OZ2_NST, tempty0 = tfull0 + 8 * OZ2_NACC;
  uint8_t *gtail = gbase + OZ2_NST * OZ2_STAGE + 16 * OZ2_NST + 16 * OZ2_NACC;
  volatile uint32_t *holder = reinterpret_cast<volatile uint32_t *>(gtail + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(gtail + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int nmtp = nmt >> 1;  // m-tile pairs (nmt is even: the A slices are padded to a pair)
  const int ntiles = 2 * nmtp * nnt;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)holder)),
                 "r"(OZ2_NACC * OZ_TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int st = 0; st < OZ2_NST; ++st) {
      mbar_init(full0 + 8 * st, 1);   // the leader's expect-tx arrive (and both CTAs' bytes)
      mbar_init(empty0 + 8 * st, 1);
    }
    for (int a = 0; a < OZ2_NACC; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 16);  // the eight epilogue warps of both CTAs
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();  // barriers of both CTAs initialised before any remote arrive
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;

  auto decode = [&](int t, int &par, int &mtp, int &nt) {
    nt = t % nnt;
    mtp = (t / nnt) % nmtp;
    par = t / (nnt * nmtp);
  };
  // the pair decides together: a tile is skipped only when none of its 256 rows runs
  auto wanted = [&](int par, int mtp, int nt) -> bool {
    if (nt * OZ_TN >= (par ? kv : ku)) return false;
    const int m0 = mtp * 2 * TM;
    if (m0 >= rows) return false;
    if (sc == nullptr) return true;
    const int r0 = m0 / rpr, r1 = (min(m0 + 2 * TM, rows) - 1) / rpr;
    for (int r = r0; r <= r1; ++r)
      if (sc[r].state == ST_RUN) return true;
    return false;
  };

  if (warp == 0) {
    if (lane == 0) {  // producer (both CTAs): per stage one K tile of its A rows and of its halves of B_j, B_j2
      const uint32_t lead_full0 = map_rank(full0, 0);
      constexpr int RA = A_TILE / OZ2_ROWB, RB = OZ_BT / OZ2_ROWB, RH = OZ2_BH / OZ2_ROWB;
      int s = 0, it = 0;
      uint32_t ph = 0;
      for (int t = pair; t < ntiles && !*abort_flag; t += npairs) {
        int par, mtp, nt;
        decode(t, par, mtp, nt);
        if (!wanted(par, mtp, nt)) continue;
        const int mt = 2 * mtp + (int)rank;
        for (int pr = 0; pr < sch.nunits && !*abort_flag; ++pr) {
          // row index (OZ2_ROWB bytes) of the unit's first A tile / B halves in the packed slice buffers
          const bool two = sch.sj2[pr] > 0;
          const int ya = (((par * NS + (sch.si[pr] - 1)) * nmt + mt) * nks) * RA;
          const int yb = (((par * NS + (sch.sj[pr] - 1)) * nnt + nt) * nks) * RB + (int)rank * RH;
          const int yb2 = (((par * NS + (max((int)sch.sj2[pr], 1) - 1)) * nnt + nt) * nks) * RB + (int)rank * RH;
          for (int kk = sch.k0[pr]; kk < sch.k1[pr]; ++kk) {
            if (it >= OZ2_NST && !mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
              atomicExch(err, 21);
              *abort_flag = 1;
              break;
            }
            const uint32_t sa = base + s * OZ2_STAGE;
            const uint32_t fb = lead_full0 + 8 * s;
            // the leader expects both CTAs' bytes of the stage
            if (rank == 0) mbar_expect_tx(full0 + 8 * s, (uint32_t)(2 * (A_TILE + (two ? 2 : 1) * OZ2_BH)));
            tma_rows2(sa, &tmA, ya + kk * RA, fb);
            tma_rows2(sa + A_TILE, &tmB, yb + kk * RB, fb);
            if (two) tma_rows2(sa + A_TILE + OZ2_BH, &tmB, yb2 + kk * RB, fb);
            ++it;
            if (++s == OZ2_NST) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {  // the leader: MMA issuer for the pair (the tile kernel's issuer)
      constexpr uint64_t DHI = ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61) | (1ull << 16);
      constexpr uint32_t B1 = A_TILE >> 4, B2 = (A_TILE + OZ2_BH) >> 4;
      int s = 0, gc = 0;
      uint32_t ph = 0;
      for (int t = pair; t < ntiles && !*abort_flag; t += npairs) {
        int par, mtp, nt;
        decode(t, par, mtp, nt);
        if (!wanted(par, mtp, nt)) continue;
        uint32_t d = 0;
        for (int pr = 0; pr < sch.nunits && !*abort_flag; ++pr) {
          const bool split = sch.split[pr] != 0, first = sch.first[pr] != 0, two = sch.sj2[pr] > 0;
          if (first) {
            bool ok = true;
            for (int q = 0; q < (split ? 2 : 1); ++q) {  // a split unit fills two accumulators
              const int acc = (gc + q) % OZ2_NACC, ause = (gc + q) / OZ2_NACC;
              if (gc + q >= OZ2_NACC && !mbar_wait_cluster(tempty0 + 8 * acc, (ause - 1) & 1)) ok = false;
            }
            if (!ok) {
              atomicExch(err, 24);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            d = tmem + (uint32_t)((gc % OZ2_NACC) * OZ_TN);
          }
          const uint32_t d2 = split ? tmem + (uint32_t)(((gc + 1) % OZ2_NACC) * OZ_TN) : d;
          const int kb = sch.k0[pr], ke = sch.k1[pr];
          for (int kk = kb; kk < ke; ++kk) {
            if (!mbar_wait(full0 + 8 * s, ph)) {
              atomicExch(err, 22);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = (base + s * OZ2_STAGE) >> 4;
            const uint32_t f1 = (first && kk == kb) ? 0u : 1u;
#pragma unroll
            for (int sub = 0; sub < TK / 16; ++sub)
              mma2_bf16(d, DHI | (sa + 2 * sub), DHI | (sa + B1 + 2 * sub), sub == 0 ? f1 : 1u);
            if (two) {
              const uint32_t f2 = split ? f1 : 1u;
#pragma unroll
              for (int sub = 0; sub < TK / 16; ++sub)
                mma2_bf16(d2, DHI | (sa + 2 * sub), DHI | (sa + B2 + 2 * sub), sub == 0 ? f2 : 1u);
            }
            commit2_both(empty0 + 8 * s);
            if (++s == OZ2_NST) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (sch.last[pr]) {
            for (int q = 0; q < (split ? 2 : 1); ++q) commit2_both(tfull0 + 8 * ((gc + q) % OZ2_NACC));
            gc += split ? 2 : 1;
          }
        }
      }
    }
  } else {  // epilogue warps 2..9 of both CTAs: their own 128 rows
    const int lg = warp & 3, h = (warp - 2) >> 2;
    const uint32_t my_tempty0 = (rank == 0) ? tempty0 : map_rank(tempty0, 0);
    int gc = 0;
    for (int t = pair; t < ntiles; t += npairs) {
      int par, mtp, nt;
      decode(t, par, mtp, nt);
      if (!wanted(par, mtp, nt)) continue;
      const int mt = 2 * mtp + (int)rank;
      const int row = mt * TM + lg * 32 + lane;
      const bool rok = row < rows;
      const int e = rok ? erow[par * (nmt * TM) + row] : 0;
      long long acci[64];
#pragma unroll
      for (int q = 0; q < 64; ++q) acci[q] = 0;
      bool stop = false;
      for (int g = 0; g < sch.ngroups; ++g) {
        const int acc = gc % OZ2_NACC, ause = gc / OZ2_NACC;
        const bool ok = mbar_wait(tfull0 + 8 * acc, ause & 1);
        __syncwarp();
        if (!ok || *abort_flag) {
          if (lane == 0 && !ok) atomicExch(err, 23);
          *abort_flag = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int gs = sch.gsh[g];
        constexpr int FIX = oz_fix(NB);
        const float up = __uint_as_float((uint32_t)(127 + (gs >= 0 ? FIX - gs : FIX)) << 23);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * OZ_TN + h * 64 + c * 16), v);
          if (gs >= 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rz(v[q] * up) << gs;
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rn(v[q] * up);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (rank == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(my_tempty0 + 8 * acc) : "memory");
          else mbar_arrive_remote(my_tempty0 + 8 * acc);
        }
        ++gc;
      }
      if (stop) break;
      if (rok) {
        const double scale = (e == OZ_EXP_NAN) ? __longlong_as_double(0x7ff8000000000000ll)
                                               : ldexp(1.0, e + eB - 2 * oz_se(NB, NS));
        const double unit = 1.0 / (double)(1LL << oz_fix(NB));
        const int kx = e + eB - 2 * oz_se(NB, NS) - oz_fix(NB);
        const int c0 = nt * OZ_TN + h * 64;
        const int ncols = min(64, (par ? kv : ku) - c0);
        const size_t o = (size_t)row * ld + par + 2 * (size_t)c0;
        oz_store(acci, ncols, e, kx, scale, unit, y + o, 2);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // neither CTA frees its tensor memory or leaves while the pair may still use it
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ2_NACC * OZ_TN) : "memory");
}

// ---------------------------------------------------------------- cluster-multicast variant
// The tile kernel's GEMM with the CTAs of a CM x CN cluster on a CM x CN block of output tiles:
// the CN CTAs of a cluster row compute tiles of the same m tile and need the same A slice tiles,
// the CM CTAs of a column the same B slice tiles.  Each K tile of a stage is read from L2 once per
// row (A) or column (B), by one of its CTAs, and multicast into the shared memory of every CTA that
// needs it (cp.async.bulk .multicast::cluster), so the cluster reads (CM + CN) / (2 CM CN) of the
// tile kernel's operand bytes from L2.  Every SM still receives a full stage per step.
// Pipeline: each CTA's "full" barrier expects the whole stage (its own copies and its peers'); its
// "empty" barrier counts the releases of every CTA its copies write into (itself, its row and its
// column: CM + CN - 1), and each CTA's MMA commit releases the stage in those same CTAs.  All CTAs
// of a cluster run the same sequence of stages (the block of tiles, its units and K tiles), so the
// stages line up; a block is skipped only when none of its tiles has work, and a CTA whose own tile
// lies outside the valid tiles (an odd column-tile count) still copies its share and stores nothing.
// Every wait is bounded; the cluster meets at a barrier before any CTA frees its tensor memory and
// exits, so no CTA leaves while a peer may still copy into it or release a stage there.
__device__ __forceinline__ void bulk_g2s_mc(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                            uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "h"(mask)
      : "memory");
}
__device__ __forceinline__ void commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                   bar),
               "h"(mask)
               : "memory");
}

template <int NB, int NS, int CM, int CN>
__global__ void __launch_bounds__(320, 1) oz_gemm_mc_kernel(const uint8_t *__restrict__ apack, size_t a_slice_bytes,
                                                            const uint8_t *__restrict__ bpack, size_t b_slice_bytes,
                                                            const int *__restrict__ erow, int eB, int nks, int nmt,
                                                            int nnt, int rows, double *__restrict__ y, int ld, int ku,
                                                            int kv, OzSched sch, const KrylovScalars *__restrict__ sc,
                                                            int rpr, int *__restrict__ err, int inv) {
  constexpr int CS = CM * CN;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  const uint32_t bars = base + OZ_NST * OZ_STAGE;
  const uint32_t full0 = bars, empty0 = bars + 8 * OZ_NST, tfull0 = bars + 16 * OZ_NST, tempty0 = tfull0 + 8 * OZ_NACC;
  volatile uint32_t *holder =
      reinterpret_cast<volatile uint32_t *>(gbase + OZ_NST * OZ_STAGE + 16 * OZ_NST + 16 * OZ_NACC + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + OZ_NST * OZ_STAGE + 16 * OZ_NST + 16 * OZ_NACC + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rank = (int)cluster_rank();
  const int ci = rank / CN, cj = rank % CN;  // this CTA's row (m) and column (n) in the block
  // multicast masks: the CTAs of this row (same A), of this column (same B), and both (releases)
  uint16_t row_mask = 0, col_mask = 0;
  for (int q = 0; q < CN; ++q) row_mask |= (uint16_t)(1u << (ci * CN + q));
  for (int q = 0; q < CM; ++q) col_mask |= (uint16_t)(1u << (q * CN + cj));
  const uint16_t rel_mask = row_mask | col_mask;
  const int cluster = blockIdx.x / CS, nclusters = gridDim.x / CS;
  const int nbm = nmt / CM, nbn = (nnt + CN - 1) / CN;  // blocks of tiles per parity (nmt is even)
  const int nblocks = 2 * nbm * nbn;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)holder)),
                 "r"(OZ_NACC * OZ_TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < OZ_NST; ++s) {
      mbar_init(full0 + 8 * s, 1);            // this CTA's expect-tx arrive; the bytes of every copy
      mbar_init(empty0 + 8 * s, CM + CN - 1);  // releases by every CTA this CTA's copies write into
    }
    for (int a = 0; a < OZ_NACC; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 8);  // one arrive per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();  // every CTA's barriers initialised before any copy or release reaches them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;

  auto decode = [&](int b, int &par, int &bm, int &bn) {
    bn = b % nbn;
    bm = (b / nbn) % nbm;
    par = b / (nbn * nbm);
  };
  auto wanted = [&](int par, int mt, int nt) -> bool {
    if (nt >= nnt || nt * OZ_TN >= ((par && !inv) ? kv : ku)) return false;
    if (mt * TM >= rows) return false;  // the padding m-tile of an odd count (A slices come in pairs)
    if (sc == nullptr) return true;
    const int m0 = mt * TM;
    const int r0 = m0 / rpr, r1 = (min(m0 + TM, rows) - 1) / rpr;
    for (int r = r0; r <= r1; ++r)
      if (sc[r].state == ST_RUN) return true;
    return false;
  };
  auto block_wanted = [&](int par, int bm, int bn) -> bool {
    for (int q = 0; q < CS; ++q)
      if (wanted(par, bm * CM + q / CN, bn * CN + q % CN)) return true;
    return false;
  };

  if (warp == 0) {
    if (lane == 0) {  // producer: this CTA's share of each stage, multicast to the CTAs that need it
      int it = 0;
      for (int b = cluster; b < nblocks && !*abort_flag; b += nclusters) {
        int par, bm, bn;
        decode(b, par, bm, bn);
        if (!block_wanted(par, bm, bn)) continue;
        const int mt = bm * CM + ci, nt = min(bn * CN + cj, nnt - 1);  // copies stay inside the slices
        for (int pr = 0; pr < sch.nunits && !*abort_flag; ++pr) {
          const uint8_t *at = apack + ((size_t)par * NS + (sch.si[pr] - 1)) * a_slice_bytes + (size_t)mt * nks * A_TILE;
          const uint8_t *bt = bpack + ((size_t)par * NS + (sch.sj[pr] - 1)) * b_slice_bytes + (size_t)nt * nks * OZ_BT;
          const int ke = sch.k1[pr];
          for (int kk = sch.k0[pr]; kk < ke; kk += OZ_KT, ++it) {
            const int kt = min(OZ_KT, ke - kk);  // K tiles in this stage
            const int s = it % OZ_NST, use = it / OZ_NST;
            if (it >= OZ_NST && !mbar_wait_cluster(empty0 + 8 * s, (use - 1) & 1)) {
              atomicExch(err, 41);
              *abort_flag = 1;
              break;
            }
            const uint32_t st = base + s * OZ_STAGE;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, (uint32_t)(kt * (A_TILE + OZ_BT)));
            for (int t = 0; t < kt; ++t) {
              if (t % CN == cj) {  // A K tile t: one copy per row
                if (CN == 1) bulk_g2s(st + t * A_TILE, at + (size_t)(kk + t) * A_TILE, A_TILE, fb);
                else bulk_g2s_mc(st + t * A_TILE, at + (size_t)(kk + t) * A_TILE, A_TILE, fb, row_mask);
              }
              if (t % CM == ci) {  // B K tile t: one copy per column
                const uint32_t dst = st + OZ_KT * A_TILE + t * OZ_BT;
                if (CM == 1) bulk_g2s(dst, bt + (size_t)(kk + t) * OZ_BT, OZ_BT, fb);
                else bulk_g2s_mc(dst, bt + (size_t)(kk + t) * OZ_BT, OZ_BT, fb, col_mask);
              }
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int it = 0, gc = 0;
      for (int b = cluster; b < nblocks && !*abort_flag; b += nclusters) {
        int par, bm, bn;
        decode(b, par, bm, bn);
        if (!block_wanted(par, bm, bn)) continue;
        uint32_t d = 0;
        for (int pr = 0; pr < sch.nunits && !*abort_flag; ++pr) {
          if (sch.first[pr]) {
            const int acc = gc % OZ_NACC, ause = gc / OZ_NACC;
            if (gc >= OZ_NACC && !mbar_wait(tempty0 + 8 * acc, (ause - 1) & 1)) {
              atomicExch(err, 42);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            d = tmem + (uint32_t)(acc * OZ_TN);
          }
          const int kb = sch.k0[pr], ke = sch.k1[pr];
          for (int kk = kb; kk < ke; kk += OZ_KT, ++it) {
            const int kt = min(OZ_KT, ke - kk);
            const int s = it % OZ_NST, use = it / OZ_NST;
            if (!mbar_wait_cluster(full0 + 8 * s, use & 1)) {
              atomicExch(err, 43);
              *abort_flag = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * OZ_STAGE;
            for (int t = 0; t < kt; ++t) {
#pragma unroll
              for (int sub = 0; sub < TK / 16; ++sub) {
                const uint32_t o = sub * 32;
                mma_bf16_n128(d, sdesc(st + t * A_TILE + o), sdesc(st + OZ_KT * A_TILE + t * OZ_BT + o),
                              (sch.first[pr] && kk == kb && t == 0 && sub == 0) ? 0u : 1u);
              }
            }
            // the stage is free again in this CTA and in the CTAs whose copies wrote into it
            if (CS == 1)
              asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                               empty0 + 8 * s)
                           : "memory");
            else
              commit_mc(empty0 + 8 * s, rel_mask);
          }
          if (sch.last[pr]) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tfull0 + 8 * (gc % OZ_NACC))
                         : "memory");
            ++gc;
          }
        }
      }
    }
  } else {  // epilogue warps 2..9
    const int lg = warp & 3, h = (warp - 2) >> 2;
    int gc = 0;
    for (int b = cluster; b < nblocks; b += nclusters) {
      int par, bm, bn;
      decode(b, par, bm, bn);
      if (!block_wanted(par, bm, bn)) continue;
      const int mt = bm * CM + ci, nt = bn * CN + cj;
      const bool mine = wanted(par, mt, nt);
      const int row = mt * TM + lg * 32 + lane;
      const bool rok = mine && row < rows;
      const int e = rok ? erow[par * (nmt * TM) + row] : 0;
      long long acci[64];
#pragma unroll
      for (int q = 0; q < 64; ++q) acci[q] = 0;
      bool stop = false;
      for (int g = 0; g < sch.ngroups; ++g) {
        const int acc = gc % OZ_NACC, ause = gc / OZ_NACC;
        const bool ok = mbar_wait(tfull0 + 8 * acc, ause & 1);
        __syncwarp();
        if (!ok) {
          if (lane == 0) atomicExch(err, 44);
          *abort_flag = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int gs = sch.gsh[g];
        constexpr int FIX = oz_fix(NB);
        const float up = __uint_as_float((uint32_t)(127 + (gs >= 0 ? FIX - gs : FIX)) << 23);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * OZ_TN + h * 64 + c * 16), v);
          if (gs >= 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rz(v[q] * up) << gs;
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) acci[c * 16 + q] += (long long)__float2int_rn(v[q] * up);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * acc) : "memory");
        ++gc;
      }
      if (stop) break;
      if (rok) {
        const double scale = (e == OZ_EXP_NAN) ? __longlong_as_double(0x7ff8000000000000ll)
                                               : ldexp(1.0, e + eB - 2 * oz_se(NB, NS));
        const double unit = 1.0 / (double)(1LL << oz_fix(NB));
        const int kx = e + eB - 2 * oz_se(NB, NS) - oz_fix(NB);
        const int c0 = nt * OZ_TN + h * 64;
        const int ncols = min(64, ((par && !inv) ? kv : ku) - c0);
        // DCT-II inverse: the even / odd mode sums E, O as [par][row][ku]; else the interleaved spectrum
        const size_t o = inv ? ((size_t)par * rows + row) * ku + c0 : (size_t)row * ld + par + 2 * (size_t)c0;
        oz_store(acci, ncols, e, kx, scale, unit, y + o, inv ? 1 : 2);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while a peer may still copy into it or release a stage there
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_NACC * OZ_TN) : "memory");
}

// Schedule of one output tile.  Exact groups: units of one weight d < tail over one K chunk (the
// longest multiple of 64 K values whose sum stays exact, kc), at most gmax units per accumulator.
// The tail (d >= tail, FP32-rounded) is cut into chunks of at most 3 pairs over the whole K range,
// each in its own accumulator, and the chunks are spread between the exact groups: every group
// costs the epilogue a pass over its accumulator, so runs of short exact groups alone would hold
// the MMA issuer waiting for accumulators, while the tail's longer groups let the epilogue catch up.
// Fused schedule (the tile kernel): pairs that share the A slice i run as one unit whose stages hold
// one K tile of A_i and of every B_j it meets, so A_i crosses into the SM once for them all (the
// operand stream into each SM is what bounds the GEMM).  Exact groups of one product each (gmax = 1)
// pair up by i into "split" units, the two products filling two consecutive groups' accumulators;
// the tail is grouped by i instead of by weight (two pairs per accumulator: products of
// different weights share an accumulator since the slices carry their scale).  The 8-bit format:
// 15 exact pairs in 6 split units and 3 single ones, 13 tail pairs in 6 units of two and 1 single;
// 44 operand K tiles per K step instead of 56.
static OzSched oz_schedule(int kpad, OzFmt f, bool fuse) {
  OzSched s{};
  const long long qmax = (f.nb == 8) ? 128 : (1LL << f.nb) - 1;  // largest digit magnitude
  const int nks = kpad / TK;
  const int kcs = std::max(1, std::min(nks, (int)((1LL << 24) / (qmax * qmax) / TK)));  // K tiles per chunk
  const long long cap = (1LL << 24) / (qmax * qmax * (long long)kcs * TK);               // units per accumulator
  const int gmax = (int)std::max(1LL, std::min(4LL, cap));
  int tail_d = (f.nb == 8) ? 7 : 8;
  for (long long k = 1024; k < kpad; k *= 2) ++tail_d;
  struct Unit {
    int i, j[2], nb, k0, k1;  // A slice i with nb (1 or 2) B slices j[] over K tiles [k0, k1)
    bool split;               // the two products fill two consecutive (exact) groups
  };
  struct Group {
    int d, d2;  // weights of its products (d2: the second group of a split unit, else 0)
    std::vector<Unit> units;
  };
  std::vector<Group> exact, tail;
  int npairs = 0;
  for (int d = 2; d <= f.ns + 1; ++d) {
    std::vector<std::pair<int, int>> pairs;
    for (int i = 1; i <= f.ns; ++i) {
      const int j = d - i;
      if (j >= 1 && j <= f.ns) pairs.push_back({i, j});
    }
    npairs += (int)pairs.size();
    if (d < tail_d) {
      for (int c0 = 0; c0 < nks; c0 += kcs) {
        const int c1 = std::min(nks, c0 + kcs);
        for (size_t q = 0; q < pairs.size(); ++q) {
          if (q % gmax == 0) exact.push_back({d, 0, {}});
          exact.back().units.push_back({pairs[q].first, {pairs[q].second, 0}, 1, c0, c1, false});
        }
      }
    } else if (!fuse) {
      for (const auto &pq : pairs) {
        if (tail.empty() || (int)tail.back().units.size() == 3) tail.push_back({tail_d, 0, {}});
        tail.back().units.push_back({pq.first, {pq.second, 0}, 1, 0, nks, false});
      }
    }
  }
  if (fuse) {
    // tail by A slice: the pairs (i, j) with tail <= i + j <= ns + 1, two per unit (one accumulator)
    for (int i = 1; i <= f.ns; ++i) {
      Unit u{i, {0, 0}, 0, 0, nks, false};
      for (int j = 1; j <= f.ns; ++j) {
        if (i + j < tail_d || i + j > f.ns + 1) continue;
        if (u.nb == 2) {
          tail.push_back({tail_d, 0, {u}});
          u.nb = 0;
        }
        u.j[u.nb++] = j;
      }
      if (u.nb > 0) tail.push_back({tail_d, 0, {u}});
    }
    // exact groups of one product: by (K chunk, i), consecutive ones paired into split units
    if (gmax == 1) {
      std::stable_sort(exact.begin(), exact.end(), [](const Group &x, const Group &y) {
        const Unit &a = x.units[0], &b = y.units[0];
        return a.k0 != b.k0 ? a.k0 < b.k0 : a.i < b.i;
      });
      std::vector<Group> fused;
      for (size_t q = 0; q < exact.size(); ++q) {
        const Unit &a = exact[q].units[0];
        if (q + 1 < exact.size() && exact[q + 1].units[0].i == a.i && exact[q + 1].units[0].k0 == a.k0) {
          const Unit &b = exact[q + 1].units[0];
          fused.push_back({exact[q].d, exact[q + 1].d, {{a.i, {a.j[0], b.j[0]}, 2, a.k0, a.k1, true}}});
          ++q;
        } else {
          fused.push_back(exact[q]);
        }
      }
      exact.swap(fused);
    }
  }
  std::vector<const Group *> order;
  const size_t ne = exact.size(), nt = tail.size();
  size_t ie = 0;
  for (size_t it = 0; it < nt; ++it) {  // spread: exact groups, a tail chunk, exact groups, ...
    const size_t upto = (it + 1) * ne / (nt + 1);
    for (; ie < upto; ++ie) order.push_back(&exact[ie]);
    order.push_back(&tail[it]);
  }
  for (; ie < ne; ++ie) order.push_back(&exact[ie]);
  const int fix = oz_fix(f.nb);
  int nu = 0, ng = 0;
  auto shift = [&](int d, bool ex) { return (int8_t)((ex && fix - f.nb * (d - 2) >= 0) ? fix - f.nb * (d - 2) : -1); };
  for (const Group *g : order) {
    const bool ex = g->d < tail_d;
    if (ng + 1 >= OZ_MAXU) throw Error(LAG_EINVAL, "exact-slice schedule: too many groups");
    s.gsh[ng] = shift(g->d, ex);
    if (g->d2 > 0) s.gsh[ng + 1] = shift(g->d2, true);
    for (size_t q = 0; q < g->units.size(); ++q) {
      if (nu >= OZ_MAXU) throw Error(LAG_EINVAL, "exact-slice schedule: too many units");
      const Unit &u = g->units[q];
      s.si[nu] = (int8_t)u.i;
      s.sj[nu] = (int8_t)u.j[0];
      s.sj2[nu] = (int8_t)(u.nb > 1 ? u.j[1] : 0);
      s.split[nu] = u.split ? 1 : 0;
      s.k0[nu] = (uint8_t)u.k0;
      s.k1[nu] = (uint8_t)u.k1;
      s.first[nu] = (q == 0);
      s.last[nu] = (q + 1 == g->units.size());
      s.ug[nu] = (uint8_t)ng;
      // a unit of two B slices takes one K tile per stage (A and both B tiles)
      s.nstage += (u.nb > 1) ? (u.k1 - u.k0) : (u.k1 - u.k0 + OZ_KT - 1) / OZ_KT;
      ++nu;
    }
    ng += (g->d2 > 0) ? 2 : 1;
  }
  s.nunits = nu;
  s.ngroups = ng;
  s.npairs = npairs;
  return s;
}

int dst_oz_products(int n) {
  const int kpad = div_up((n + 1) / 2, TK) * TK;
  return oz_schedule(kpad, oz_format(kpad), false).npairs;
}

bool dst_oz_supported(int n) {
  const int ku = (n + 1) / 2;
  const int kpad = div_up(ku, TK) * TK;
  return n >= 16 && 63LL * 63LL * kpad <= (1LL << 24);  // one pair per accumulator at least
}

size_t dst_oz_bytes(int n, int kind) {
  const int ku = (n + 1) / 2;
  return (kind == 1 ? 2 : 1) * 2 * (size_t)OZ_SMAX * div_up(ku, OZ_TN) * div_up(ku, TK) * OZ_BT;
}

void dst_build_oz(DstPlan &dp, DevBuf &store, size_t off, cudaStream_t s) {
  const int nks = div_up(dp.ku, TK), nnt = div_up(dp.ku, OZ_TN);
  dp.kpad_u = nks;
  dp.npad_u = nnt;
  dp.oz_slice_bytes = (size_t)nnt * nks * OZ_BT;
  dp.oz_b = store.as<uint8_t>() + off;
  int eB = 0;
  // every |S| <= sqrt(2 / (n + 1)) < 2^eB (DST-I); every |V| <= sqrt(2 / n) < 2^eB (DCT-II)
  frexp(std::sqrt(2.0 / (double)(dp.kind == 1 ? dp.n : dp.n + 1)), &eB);
  dp.oz_eB = eB;
  const OzFmt f = oz_format(nks * TK);
  dp.oz_nb = f.nb;
  dp.oz_ns = f.ns;
  dim3 g(div_up(nks * TK, 128), nnt * OZ_TN, 2);
  auto pack_b = [&](const double *m0, int k0n, int n0n, int ld0, const double *m1, int k1n, int n1n, int ld1,
                    uint8_t *out) {
    if (f.nb == 8)
      oz_pack_b_kernel<8, 7><<<g, 128, 0, s>>>(m0, k0n, n0n, ld0, m1, k1n, n1n, ld1, nks, nnt, eB, out,
                                               dp.oz_slice_bytes);
    else if (f.nb == 7)
      oz_pack_b_kernel<7, 8><<<g, 128, 0, s>>>(m0, k0n, n0n, ld0, m1, k1n, n1n, ld1, nks, nnt, eB, out,
                                               dp.oz_slice_bytes);
    else
      oz_pack_b_kernel<6, 9><<<g, 128, 0, s>>>(m0, k0n, n0n, ld0, m1, k1n, n1n, ld1, nks, nnt, eB, out,
                                               dp.oz_slice_bytes);
    count_launch();
    LAG_LAUNCH_CHECK();
  };
  pack_b(dp.su, dp.ku, dp.ku, dp.ku, dp.sv, dp.kv, dp.kv, dp.kv, dp.oz_b);
  if (dp.kind == 1) {  // inverse operands: even / odd input modes x ceil(n/2) output columns
    dp.oz_bi = dp.oz_b + 2 * (size_t)f.ns * dp.oz_slice_bytes;
    pack_b(dp.ie, dp.ku, dp.ku, dp.ku, dp.io, dp.kv, dp.ku, dp.ku, dp.oz_bi);
  }
  dp.oz = true;
}

// 2-D tensor map over `nrows` rows of 128 bytes (64 bf16) at base: TMA copies of box_rows whole
// rows, verbatim (the tiles are already in the swizzled shared-memory layout)
// The driver's tensor-map encoder, looked up through the runtime (the library does not link the
// driver library, so it still loads where no driver is installed)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (fn == nullptr) throw Error(LAG_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// a buffer of pre-swizzled tiles as rows of OZ2_ROWB bytes (256 8-byte elements): a tile copy is
// one box of whole rows, which the copy engine moves as a few long requests instead of one per
// 128-byte row
static CUtensorMap rows_map(const void *base, uint64_t nrows, uint32_t box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {OZ2_ROWB / 8, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {OZ2_ROWB};
  const cuuint32_t box[2] = {OZ2_ROWB / 8, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = tensor_map_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims,
                                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(LAG_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// m-tiles of packed A slices: rounded up to a pair for the two-SM GEMM
static int oz_mtiles(int rows) {
  const int nmt = div_up(rows, TM);
  return nmt + (nmt & 1);
}

// the two-SM variant is opt-in (LAGWAVE_OZ_PAIR=1): it streams a third fewer operand bytes per SM
// but measured slower than the one-SM kernel (133 against 113 us at a 1024 x 2048 transform: a
// pair's stage completes only when both SMs' copies have landed on the leader's barrier, and the
// SMs then receive 29 instead of 49 bytes per clock)
static bool oz_pair_enabled() {
  const char *v = std::getenv("LAGWAVE_OZ_PAIR");
  return v != nullptr && v[0] == '1';
}

// SMs of the current device, read once per device
static int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  LAG_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(LAG_EINVAL, "device ordinal out of range");
  int n = cache[dev].load();
  if (n == 0) {
    LAG_CUDA_CHECK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    cache[dev].store(n);
  }
  return n;
}
// CTAs of a stream-K launch: one per SM
static int oz_sk_ctas() { return std::min(device_sms(), OZ_SK_MAXG); }
// stream-K is opt-in (LAGWAVE_OZ_SK=1): with every SM on its own range the CTAs no longer read the
// same operand lines at the same time, the L2 serves every copy separately, and the kernel measured
// slower than the tile kernel on 24 fewer SMs (178.6 against 143.3 us at 2048 modes x 1024 rows)
static bool oz_sk_enabled() {
  const char *v = std::getenv("LAGWAVE_OZ_SK");
  return v != nullptr && v[0] == '1';
}

// scratch layout: the stream-K area first, at a place that does not move with the row count
// [control 256 B][flags G x 8 ints, to 256 B][parts G x TM x TN int64], then [A slices][row
// exponents] | 256-aligned [E / O sums (DCT-II inverse)]
static size_t oz_sk_flag_bytes(int G) { return ((size_t)G * 8 * sizeof(int) + 255) & ~(size_t)255; }
static size_t oz_sk_bytes() {
  const int G = oz_sk_ctas();
  return 256 + oz_sk_flag_bytes(G) + (size_t)G * TM * OZ_TN * sizeof(long long);
}

size_t dst_oz_scratch_bytes(const DstPlan &dp, int rows) {
  const size_t nmt = oz_mtiles(rows);
  const size_t eo = (dp.kind == 1) ? 2 * (size_t)rows * dp.ku * sizeof(double) + 256 : 0;  // DCT-II E / O sums
  return oz_sk_bytes() + 2 * (size_t)OZ_SMAX * nmt * dp.kpad_u * A_TILE + 2 * nmt * TM * sizeof(int) + 256 + eo;
}

// DCT-II inverse butterfly: x[k] = E[k] + O[k], x[n-1-k] = E[k] - O[k] (k < ceil(n/2)); rows of
// finished right-hand sides are left as they are (their GEMM tiles were skipped).
__global__ void oz_butterfly_kernel(const double *__restrict__ eo, double *__restrict__ x, int rows, int n, int ku,
                                    const KrylovScalars *__restrict__ sc, int rpr) {
  const int row = blockIdx.x;  // one block per row
  if (row >= rows || (sc != nullptr && sc[row / rpr].state != ST_RUN)) return;
  const double *E = eo + (size_t)row * ku, *O = eo + ((size_t)rows + row) * ku;
  double *xr = x + (size_t)row * n;
  for (int k = threadIdx.x; k < ku; k += blockDim.x) {
    const double e = E[k], o = O[k];
    xr[k] = e + o;
    if (n - 1 - k != k) xr[n - 1 - k] = e - o;
  }
}

// cluster shape of the multicast kernel: LAGWAVE_OZ_CLUSTER=2x2 / 1x2 / 2x1 (rows x columns of
// tiles), else 0 x 0 (not used)
static void oz_cluster_shape(int &cm, int &cn) {
  cm = cn = 0;
  const char *v = std::getenv("LAGWAVE_OZ_CLUSTER");
  if (v == nullptr || (v[0] != '1' && v[0] != '2') || v[1] != 'x' || (v[2] != '1' && v[2] != '2') || v[3] != 0) return;
  cm = v[0] - '0';
  cn = v[2] - '0';
  if (cm * cn == 1) cm = cn = 0;
}

// the GEMM kernel of a forward (inv = 0) or DCT-II inverse (inv = 1) transform of `rows` rows,
// rpr rows per right-hand side
int dst_oz_gemm_variant(const DstPlan &dp, int rows, int rpr, int inv) {
  const size_t a_slice = (size_t)oz_mtiles(rows) * dp.kpad_u * A_TILE;
  // TMA coordinates are signed 32-bit: the pair kernel addresses the slice buffers by OZ2_ROWB-byte row
  if (!inv && oz_pair_enabled() && 2ull * dp.oz_ns * a_slice / OZ2_ROWB < (1ull << 31)) return OZ_GEMM_PAIRS;
  int cm, cn;
  oz_cluster_shape(cm, cn);
  if (cm > 0) return OZ_GEMM_CLUSTER;
  // tiles that run: m tiles of the rows (not the padding one) x column tiles of each parity
  const int vtiles = div_up(rows, TM) * (div_up(dp.ku, OZ_TN) + div_up(dp.kv, OZ_TN));
  const int g = oz_sk_ctas();
  // one right-hand side whose tiles leave SMs idle in the last wave: equal ranges of steps per SM
  // (at least half as many tiles as SMs: a tile is then shared by three CTAs at most)
  if (!inv && rows <= rpr && oz_sk_enabled() && vtiles % g != 0 && 2 * vtiles >= g && vtiles < 4 * g)
    return OZ_GEMM_STREAMK;
  return OZ_GEMM_TILES;
}

// the multicast kernel on CM x CN clusters: as many clusters as fit at once (at most one per block
// of tiles), each walking the blocks persistently
template <int NB, int NS, int CM, int CN>
static void oz_launch_mc(const uint8_t *apack, size_t a_slice, const uint8_t *bpack, const DstPlan &dp, const int *erow,
                         int nks, int nmt, int nnt, int rows, double *y, const OzSched &sch, const KrylovScalars *sc,
                         int rpr, int inv, cudaStream_t s) {
  static PerDeviceOnce attr;
  static std::atomic<int> fit[64];
  int dev = 0;
  LAG_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(LAG_EINVAL, "device ordinal out of range");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CM * CN;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(320, 1, 1);
  cfg.dynamicSmemBytes = OZ_SMEM;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  attr.run([&] {
    LAG_CUDA_CHECK(cudaFuncSetAttribute(oz_gemm_mc_kernel<NB, NS, CM, CN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        OZ_SMEM));
  });
  if (fit[dev].load() == 0) {
    int n = 0;
    cfg.gridDim = dim3(CM * CN, 1, 1);
    LAG_CUDA_CHECK(cudaOccupancyMaxActiveClusters(&n, oz_gemm_mc_kernel<NB, NS, CM, CN>, &cfg));
    if (n < 1) throw Error(LAG_ECUDA, "exact-slice GEMM: no cluster of this shape fits on the device");
    fit[dev].store(n);
  }
  const int nblocks = 2 * (nmt / CM) * ((nnt + CN - 1) / CN);
  cfg.gridDim = dim3(CM * CN * std::min(nblocks, fit[dev].load()), 1, 1);
  LAG_CUDA_CHECK(cudaLaunchKernelEx(&cfg, oz_gemm_mc_kernel<NB, NS, CM, CN>, apack, a_slice, bpack, dp.oz_slice_bytes,
                                    erow, dp.oz_eB, nks, nmt, nnt, rows, y, dp.n, dp.ku, dp.kv, sch, sc, rpr, dp.tc_err,
                                    inv));
}

template <int NB, int NS>
static void oz_apply_fmt(const DstPlan &dp, const double *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                         cudaStream_t s, int inv) {
  static PerDeviceOnce attr;
  attr.run([] {
    LAG_CUDA_CHECK(cudaFuncSetAttribute(oz_gemm_kernel<NB, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZT_SMEM));
    LAG_CUDA_CHECK(cudaFuncSetAttribute(oz_gemm2_kernel<NB, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ2_SMEM));
    LAG_CUDA_CHECK(cudaFuncSetAttribute(oz_gemm_sk_kernel<NB, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    LAG_CUDA_CHECK(cudaFuncSetAttribute(oz_pack_a_kernel<NB, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)oz_pack_smem(OZ_PACK_MAXK / TK + 1)));
  });
  const int nks = dp.kpad_u, nnt = dp.npad_u, nmt = oz_mtiles(rows);
  const size_t a_slice = (size_t)nmt * nks * A_TILE;
  uint8_t *apack = dp.tc_scratch + oz_sk_bytes();
  int *erow = reinterpret_cast<int *>(apack + 2 * (size_t)NS * a_slice);
  const size_t pack_smem = oz_pack_smem(nks);
  oz_pack_a_kernel<NB, NS><<<nmt * TM, OZ_PACK_THREADS, pack_smem, s>>>(x, rows, dp.n, dp.ku, dp.kv, nks, nmt, apack,
                                                                         a_slice, erow, sc, rpr, inv);
  count_launch();
  LAG_LAUNCH_CHECK();
  const int variant = dst_oz_gemm_variant(dp, rows, rpr, inv);
  const OzSched sch = oz_schedule(nks * TK, OzFmt{NB, NS}, variant == OZ_GEMM_TILES || variant == OZ_GEMM_PAIRS);
  const int ntiles = 2 * nmt * nnt;
  const int grid = std::min(ntiles, 152);
  // E / O sums of the inverse: after the packed A slices and the row exponents, 256-byte aligned
  double *eo = reinterpret_cast<double *>(
      (reinterpret_cast<uintptr_t>(erow + 2 * (size_t)nmt * TM) + 255) & ~(uintptr_t)255);
  if (variant == OZ_GEMM_PAIRS) {
    // two-SM pairs: 256-row tile pairs x column tiles x both parities, at most one pair per two SMs
    const int pairs = std::min(2 * (nmt / 2) * nnt, 76);
    const CUtensorMap tmA = rows_map(apack, 2ull * NS * a_slice / OZ2_ROWB, A_TILE / OZ2_ROWB);
    const CUtensorMap tmB = rows_map(dp.oz_b, 2ull * NS * dp.oz_slice_bytes / OZ2_ROWB, OZ2_BH / OZ2_ROWB);
    oz_gemm2_kernel<NB, NS><<<2 * pairs, 320, OZ2_SMEM, s>>>(tmA, tmB, erow, dp.oz_eB, nks, nmt, nnt, rows, y, dp.n,
                                                             dp.ku, dp.kv, sch, sc, rpr, dp.tc_err);
  } else if (variant == OZ_GEMM_CLUSTER) {
    int cm, cn;
    oz_cluster_shape(cm, cn);
    const uint8_t *bp = inv ? dp.oz_bi : dp.oz_b;
    double *yo = inv ? eo : y;
    if (cm == 2 && cn == 2)
      oz_launch_mc<NB, NS, 2, 2>(apack, a_slice, bp, dp, erow, nks, nmt, nnt, rows, yo, sch, sc, rpr, inv, s);
    else if (cm == 1)
      oz_launch_mc<NB, NS, 1, 2>(apack, a_slice, bp, dp, erow, nks, nmt, nnt, rows, yo, sch, sc, rpr, inv, s);
    else
      oz_launch_mc<NB, NS, 2, 1>(apack, a_slice, bp, dp, erow, nks, nmt, nnt, rows, yo, sch, sc, rpr, inv, s);
  } else if (variant == OZ_GEMM_STREAMK) {
    const int gsk = oz_sk_ctas();
    uint8_t *area = dp.tc_scratch;
    OzSkArea ska;
    ska.ctl = reinterpret_cast<int *>(area);
    ska.flag = reinterpret_cast<int *>(area + 256);
    ska.part = reinterpret_cast<long long *>(area + 256 + oz_sk_flag_bytes(gsk));
    oz_gemm_sk_kernel<NB, NS><<<gsk, 320, OZ_SMEM, s>>>(apack, a_slice, dp.oz_b, dp.oz_slice_bytes, erow, dp.oz_eB,
                                                        nks, nmt, nnt, rows, y, dp.n, dp.ku, dp.kv, sch, sc,
                                                        dp.tc_err, ska);
  } else {
    oz_gemm_kernel<NB, NS><<<grid, 320, OZT_SMEM, s>>>(apack, a_slice, inv ? dp.oz_bi : dp.oz_b, dp.oz_slice_bytes,
                                                      erow, dp.oz_eB, nks, nmt, nnt, rows, inv ? eo : y, dp.n, dp.ku,
                                                      dp.kv, sch, sc, rpr, dp.tc_err, inv);
  }
  count_launch();
  LAG_LAUNCH_CHECK();
  if (inv) {
    oz_butterfly_kernel<<<rows, 256, 0, s>>>(eo, y, rows, dp.n, dp.ku, sc, rpr);
    count_launch();
    LAG_LAUNCH_CHECK();
  }
}

void dst_apply_oz(const DstPlan &dp, const double *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                  cudaStream_t s, bool inverse) {
  if (rows <= 0) return;
  ProfScope prof(KC_DST64, s);
  const int inv = (inverse && dp.kind == 1) ? 1 : 0;
  if (dp.oz_nb == 8) oz_apply_fmt<8, 7>(dp, x, y, rows, rpr, sc, s, inv);
  else if (dp.oz_nb == 7) oz_apply_fmt<7, 8>(dp, x, y, rows, rpr, sc, s, inv);
  else oz_apply_fmt<6, 9>(dp, x, y, rows, rpr, sc, s, inv);
}

}  // namespace lag
