// Orthonormal DST-I along x as two folded dense GEMMs (the preconditioner's x-direction step).
//
// Sec. 2.4 inverts the Laplace preconditioner by separation of variables; the transform along x
// (FFTW in the paper, Sec. 3.1) diagonalises the Dirichlet second difference.  With
//     S[j][k] = sqrt(2/(n+1)) sin(pi (j+1)(k+1)/(n+1)),   S^2 = I,
// and S[n-1-j][k] = (-1)^k S[j][k], every row transform y = S x splits into
//     y[2k']   = sum_{j' < ceil(n/2)}  S[j'][2k']   u[j'],   u[j'] = x[j'] + x[n-1-j']  (middle once)
//     y[2k'+1] = sum_{j' < floor(n/2)} S[j'][2k'+1] v[j'],   v[j'] = x[j'] - x[n-1-j']
// i.e. two (n/2 x n/2) GEMMs over all rows at half the flops of the direct product.  The fold is
// applied while the A tile is staged into shared memory.  n + 1 has large prime factors at the
// workload sizes (2049 = 3 * 683), so the dense product is used rather than a fast transform.
//
// The cylindrical problem (Sec. 2.3 mesh, zero-flux faces at both ends of z) is diagonalised along
// z by the orthonormal DCT-II, V[k][q] = c_q cos(pi q (k + 1/2) / n) (c_0 = sqrt(1/n), else
// sqrt(2/n)).  V[n-1-k][q] = (-1)^q V[k][q], so the forward transform y = V^T x folds exactly like
// the DST (su = V[j'][2k'], sv = V[j'][2k'+1]).  V is not symmetric: the inverse x = V y gathers
// the even and the odd modes, E[k] = sum V[k][2q'] y[2q'], O[k] = sum V[k][2q'+1] y[2q'+1]
// (k < ceil(n/2)), and writes x[k] = E + O, x[n-1-k] = E - O.
#include "internal.h"

namespace lag {

// ------------------------------------------------------------------------------ matrices
__global__ void dst_matrix_kernel(int n, int ku, int kv, double *su, double *sv, float *suf, float *svf) {
  const int kp = blockIdx.x * blockDim.x + threadIdx.x;  // output column k' (fastest)
  const int jp = blockIdx.y;                             // input row j'
  const double scale = sqrt(2.0 / (double)(n + 1));
  const long long period = 2LL * (n + 1);
  if (kp < ku && jp < ku) {
    const long long m = ((long long)(jp + 1) * (long long)(2 * kp + 1)) % period;
    const double v = scale * sinpi((double)m / (double)(n + 1));
    su[(size_t)jp * ku + kp] = v;
    suf[(size_t)jp * ku + kp] = (float)v;
  }
  if (kp < kv && jp < kv) {
    const long long m = ((long long)(jp + 1) * (long long)(2 * kp + 2)) % period;
    const double v = scale * sinpi((double)m / (double)(n + 1));
    sv[(size_t)jp * kv + kp] = v;
    svf[(size_t)jp * kv + kp] = (float)v;
  }
}

void dst_build_tc(DstPlan &dp, DevBuf &store, size_t offset_bytes, cudaStream_t s);
size_t dst_tc_bytes(int n);
void dst_build_oz(DstPlan &dp, DevBuf &store, size_t offset_bytes, cudaStream_t s);
size_t dst_oz_bytes(int n, int kind);

// DCT-II halves: su[j'][k'] = V[j'][2k'] (ku x ku), sv[j'][k'] = V[j'][2k'+1] (kv x kv), and the
// inverse operands ie[q'][k] = V[k][2q'] (ku x ku), io[q'][k] = V[k][2q'+1] (kv x ku).  Angles are
// reduced exactly in integers: V[k][q] = c_q cospi(m / (2n)), m = q (2k + 1) mod 4n.
__device__ __forceinline__ double dct_entry(int n, int k, int q) {
  const long long m = ((long long)q * (long long)(2 * k + 1)) % (4LL * n);
  const double c = (q == 0) ? sqrt(1.0 / (double)n) : sqrt(2.0 / (double)n);
  return c * cospi((double)m / (2.0 * (double)n));
}

__global__ void dct_matrix_kernel(int n, int ku, int kv, double *su, double *sv, float *suf, float *svf, double *ie,
                                  double *io, float *ief, float *iof) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;  // fastest index
  const int b = blockIdx.y;
  if (a < ku && b < ku) {
    const double v = dct_entry(n, b, 2 * a);             // su[j' = b][k' = a]
    su[(size_t)b * ku + a] = v;
    suf[(size_t)b * ku + a] = (float)v;
    const double w = dct_entry(n, a, 2 * b);             // ie[q' = b][k = a]
    ie[(size_t)b * ku + a] = w;
    ief[(size_t)b * ku + a] = (float)w;
  }
  if (a < kv && b < kv) {
    const double v = dct_entry(n, b, 2 * a + 1);         // sv[j' = b][k' = a]
    sv[(size_t)b * kv + a] = v;
    svf[(size_t)b * kv + a] = (float)v;
  }
  if (a < ku && b < kv) {
    const double w = dct_entry(n, a, 2 * b + 1);         // io[q' = b][k = a]
    io[(size_t)b * ku + a] = w;
    iof[(size_t)b * ku + a] = (float)w;
  }
}

void dst_build(DstPlan &dp, DevBuf &store, int n, int tc_mode, cudaStream_t s, int kind) {
  dp.kind = kind;
  dp.n = n;
  dp.ku = (n + 1) / 2;
  dp.kv = n / 2;
  const size_t nu = (size_t)dp.ku * dp.ku, nv = (size_t)dp.kv * dp.kv;
  const size_t ninv = (kind == 1) ? nu + (size_t)dp.kv * dp.ku : 0;
  size_t bytes = (nu + nv + ninv) * (sizeof(double) + sizeof(float)) + 256;
  const size_t tc_off = (bytes + 1023) & ~(size_t)1023;
  if (tc_mode == 1) bytes = tc_off + dst_tc_bytes(n) + 256;  // + error word at the end
  if (tc_mode == 2) bytes = tc_off + dst_oz_bytes(n, kind) + 256;
  store.alloc(store.ctx, bytes, true);
  char *base = store.as<char>();
  dp.su = reinterpret_cast<double *>(base);
  dp.sv = dp.su + nu;
  dp.ie = dp.sv + nv;
  dp.io = dp.ie + (kind == 1 ? nu : 0);
  dp.su_f = reinterpret_cast<float *>(dp.sv + nv + ninv);
  dp.sv_f = dp.su_f + nu;
  dp.ie_f = dp.sv_f + nv;
  dp.io_f = dp.ie_f + (kind == 1 ? nu : 0);
  if (kind != 1) {
    dp.ie = dp.io = nullptr;
    dp.ie_f = dp.io_f = nullptr;
  }
  dim3 grid((dp.ku + 127) / 128, dp.ku > 0 ? dp.ku : 1);
  if (kind == 1)
    dct_matrix_kernel<<<grid, 128, 0, s>>>(n, dp.ku, dp.kv, dp.su, dp.sv, dp.su_f, dp.sv_f, dp.ie, dp.io, dp.ie_f,
                                           dp.io_f);
  else
    dst_matrix_kernel<<<grid, 128, 0, s>>>(n, dp.ku, dp.kv, dp.su, dp.sv, dp.su_f, dp.sv_f);
  count_launch();
  LAG_LAUNCH_CHECK();
  if (tc_mode == 1) dst_build_tc(dp, store, tc_off, s);
  if (tc_mode == 2) dst_build_oz(dp, store, tc_off, s);
}

// ------------------------------------------------------------------------------ SIMT GEMM
// One launch covers both parities (blockIdx.z).  Tile BM x BN x 16, 256 threads, each thread a
// (BM/16) x (BN/16) block of outputs.  The tile is picked per launch so that the number of tiles
// spreads evenly over the 152 SMs (float64 is ALU-bound: the tail wave is what costs).
constexpr int BK = 16;

template <int BM>
__device__ __forceinline__ bool tile_all_done(const KrylovScalars *sc, int m0, int rows, int rpr) {
  if (sc == nullptr) return false;
  const int r0 = m0 / rpr, r1 = (min(m0 + BM, rows) - 1) / rpr;
  for (int r = r0; r <= r1; ++r)
    if (sc[r].state == ST_RUN) return false;
  return true;
}

template <typename TI, typename TO, typename TA, int BM, int BN>
__global__ void __launch_bounds__(256) dst_simt_kernel(const TI *__restrict__ X, TO *__restrict__ Y, int rows, int n,
                                                       const TA *__restrict__ Su, const TA *__restrict__ Sv,
                                                       int ku, int kv, const KrylovScalars *__restrict__ sc, int rpr,
                                                       int rscale) {
  constexpr int UM = BM / 16, UN = BN / 16;       // outputs per thread
  constexpr int LA = BM * BK / 256, LB = BK * BN / 256;  // tile elements per thread
  const int parity = blockIdx.z;
  const int K = parity ? kv : ku;
  const TA *B = parity ? Sv : Su;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  if (n0 >= K || tile_all_done<BM>(sc, m0, rows, rpr)) return;
  // rscale 1: scale the input rows by 2^-e (float64 in); 2: the output rows by 2^e (float64 out)
  const bool scaled = rscale != 0 && sc != nullptr;
  int in_exp[LA];
#pragma unroll
  for (int e = 0; e < LA; ++e) {
    const int row = m0 + (threadIdx.x + e * 256) / BK;
    in_exp[e] = (scaled && rscale == 1 && row < rows) ? -residual_exponent(sc, row / rpr) : 0;
  }
  __shared__ __align__(16) TA As[BK][BM + 4];
  __shared__ __align__(16) TA Bs[BK][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  TA acc[UM][UN];
#pragma unroll
  for (int i = 0; i < UM; ++i)
#pragma unroll
    for (int j = 0; j < UN; ++j) acc[i][j] = TA(0);
  const bool odd_n = (n & 1) != 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      const int idx = tid + e * 256;
      const int r = idx / BK, kk = idx % BK;
      const int row = m0 + r, j = k0 + kk;
      TA v = TA(0);
      if (row < rows && j < K) {
        const TI *xr = X + (size_t)row * n;
        const double d1 = (double)xr[j], d2 = (double)xr[n - 1 - j];
        const TA x1 = (TA)(in_exp[e] != 0 ? scale_pow2(d1, in_exp[e]) : d1);
        const TA x2 = (TA)(in_exp[e] != 0 ? scale_pow2(d2, in_exp[e]) : d2);
        if (parity == 0) v = (odd_n && j == K - 1) ? x1 : x1 + x2;
        else v = x1 - x2;
      }
      As[kk][r] = v;
    }
#pragma unroll
    for (int e = 0; e < LB; ++e) {
      const int idx = tid + e * 256;
      const int kb = idx / BN, c = idx % BN;
      Bs[kb][c] = (k0 + kb < K && n0 + c < K) ? B[(size_t)(k0 + kb) * K + n0 + c] : TA(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA a[UM], b[UN];
#pragma unroll
      for (int i = 0; i < UM; ++i) a[i] = As[kk][ty * UM + i];
#pragma unroll
      for (int j = 0; j < UN; ++j) b[j] = Bs[kk][tx * UN + j];
#pragma unroll
      for (int i = 0; i < UM; ++i)
#pragma unroll
        for (int j = 0; j < UN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < UM; ++i) {
    const int row = m0 + ty * UM + i;
    if (row >= rows) continue;
    const int oe = (scaled && rscale == 2) ? residual_exponent(sc, row / rpr) : 0;
#pragma unroll
    for (int j = 0; j < UN; ++j) {
      const int col = n0 + tx * UN + j;
      if (col < K) Y[(size_t)row * n + 2 * col + parity] = (TO)(oe != 0 ? scale_pow2((double)acc[i][j], oe) : (double)acc[i][j]);
    }
  }
}

// fraction of the last wave that is busy when `tiles` equal tiles run over the SMs
static double wave_efficiency(long long tiles) {
  const long long sms = 152;
  const long long waves = (tiles + sms - 1) / sms;
  return waves ? (double)tiles / (double)(waves * sms) : 1.0;
}

template <typename TI, typename TO, typename TA>
static void dst_simt_launch(const DstPlan &dp, const TI *x, TO *y, int rows, int rpr, const TA *su, const TA *sv,
                            const KrylovScalars *sc, cudaStream_t s, int cls, int rscale = 0) {
  if (rows <= 0 || dp.n <= 0) return;
  ProfScope prof(cls, s);
  const int nz = dp.kv > 0 ? 2 : 1;
  auto tiles = [&](int bm, int bn) {
    return (long long)((dp.ku + bn - 1) / bn) * ((rows + bm - 1) / bm) * nz;
  };
  // largest tile whose tail wave keeps >= 90 % of the SMs busy (smaller tiles cost reuse)
  int choice = 0;
  if (wave_efficiency(tiles(64, 64)) < 0.9) choice = (wave_efficiency(tiles(64, 32)) >= 0.9) ? 1 : 2;
  if (choice == 0) {
    dim3 grid((dp.ku + 63) / 64, (rows + 63) / 64, nz);
    dst_simt_kernel<TI, TO, TA, 64, 64><<<grid, 256, 0, s>>>(x, y, rows, dp.n, su, sv, dp.ku, dp.kv, sc, rpr, rscale);
  } else if (choice == 1) {
    dim3 grid((dp.ku + 31) / 32, (rows + 63) / 64, nz);
    dst_simt_kernel<TI, TO, TA, 64, 32><<<grid, 256, 0, s>>>(x, y, rows, dp.n, su, sv, dp.ku, dp.kv, sc, rpr, rscale);
  } else {
    dim3 grid((dp.ku + 31) / 32, (rows + 31) / 32, nz);
    dst_simt_kernel<TI, TO, TA, 32, 32><<<grid, 256, 0, s>>>(x, y, rows, dp.n, su, sv, dp.ku, dp.kv, sc, rpr, rscale);
  }
  count_launch();
  LAG_LAUNCH_CHECK();
}

// Inverse DCT-II: one CTA computes the even-mode sum E and the odd-mode sum O of a BM x BN output
// tile (k < ku) and writes the butterfly x[k] = E + O, x[n-1-k] = E - O.
template <typename TI, typename TO, typename TA, int BM, int BN>
__global__ void __launch_bounds__(256) dct_inv_simt_kernel(const TI *__restrict__ Yin, TO *__restrict__ X, int rows,
                                                           int n, const TA *__restrict__ Ie, const TA *__restrict__ Io,
                                                           int ku, int kv, const KrylovScalars *__restrict__ sc,
                                                           int rpr, int rscale) {
  constexpr int UM = BM / 16, UN = BN / 16;
  constexpr int LA = BM * BK / 256, LB = BK * BN / 256;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  if (n0 >= ku || tile_all_done<BM>(sc, m0, rows, rpr)) return;
  __shared__ __align__(16) TA As[BK][BM + 4];
  __shared__ __align__(16) TA Bs[BK][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  TA acc[2][UM][UN];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int i = 0; i < UM; ++i)
#pragma unroll
      for (int j = 0; j < UN; ++j) acc[p][i][j] = TA(0);
#pragma unroll
  for (int parity = 0; parity < 2; ++parity) {
    const int K = parity ? kv : ku;   // modes of this parity
    const TA *B = parity ? Io : Ie;   // [K][ku]
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
      for (int e = 0; e < LA; ++e) {
        const int idx = tid + e * 256;
        const int r = idx / BK, kk = idx % BK;
        const int row = m0 + r, q = k0 + kk;
        As[kk][r] = (row < rows && q < K) ? (TA)Yin[(size_t)row * n + 2 * q + parity] : TA(0);
      }
#pragma unroll
      for (int e = 0; e < LB; ++e) {
        const int idx = tid + e * 256;
        const int kb = idx / BN, c = idx % BN;
        Bs[kb][c] = (k0 + kb < K && n0 + c < ku) ? B[(size_t)(k0 + kb) * ku + n0 + c] : TA(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        TA a[UM], b[UN];
#pragma unroll
        for (int i = 0; i < UM; ++i) a[i] = As[kk][ty * UM + i];
#pragma unroll
        for (int j = 0; j < UN; ++j) b[j] = Bs[kk][tx * UN + j];
#pragma unroll
        for (int i = 0; i < UM; ++i)
#pragma unroll
          for (int j = 0; j < UN; ++j) acc[parity][i][j] = fma(a[i], b[j], acc[parity][i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < UM; ++i) {
    const int row = m0 + ty * UM + i;
    if (row >= rows) continue;
    const int oe = (rscale == 2 && sc != nullptr) ? residual_exponent(sc, row / rpr) : 0;
#pragma unroll
    for (int j = 0; j < UN; ++j) {
      const int col = n0 + tx * UN + j;
      if (col >= ku) continue;
      const TA e = acc[0][i][j], o = acc[1][i][j];
      const double p1 = (double)(e + o), p2 = (double)(e - o);
      X[(size_t)row * n + col] = (TO)(oe != 0 ? scale_pow2(p1, oe) : p1);
      if (n - 1 - col != col) X[(size_t)row * n + n - 1 - col] = (TO)(oe != 0 ? scale_pow2(p2, oe) : p2);
    }
  }
}

template <typename TI, typename TO, typename TA>
static void dct_inv_launch(const DstPlan &dp, const TI *y, TO *x, int rows, int rpr, const TA *ie, const TA *io,
                           const KrylovScalars *sc, cudaStream_t s, int cls, int rscale = 0) {
  if (rows <= 0 || dp.n <= 0) return;
  ProfScope prof(cls, s);
  auto tiles = [&](int bm, int bn) { return (long long)((dp.ku + bn - 1) / bn) * ((rows + bm - 1) / bm); };
  if (wave_efficiency(tiles(64, 64)) >= 0.9) {
    dim3 grid((dp.ku + 63) / 64, (rows + 63) / 64);
    dct_inv_simt_kernel<TI, TO, TA, 64, 64><<<grid, 256, 0, s>>>(y, x, rows, dp.n, ie, io, dp.ku, dp.kv, sc, rpr,
                                                                  rscale);
  } else {
    dim3 grid((dp.ku + 31) / 32, (rows + 31) / 32);
    dct_inv_simt_kernel<TI, TO, TA, 32, 32><<<grid, 256, 0, s>>>(y, x, rows, dp.n, ie, io, dp.ku, dp.kv, sc, rpr,
                                                                  rscale);
  }
  count_launch();
  LAG_LAUNCH_CHECK();
}

void dst_inverse_f64_simt(const DstPlan &dp, const double *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                          cudaStream_t s) {
  if (dp.kind == 1) dct_inv_launch<double, double, double>(dp, x, y, rows, rpr, dp.ie, dp.io, sc, s, KC_DST64);
  else dst_apply_f64_simt(dp, x, y, rows, rpr, sc, s);
}
void dst_inverse_f64(const DstPlan &dp, const double *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                     cudaStream_t s) {
  if (dp.kind == 1 && dp.oz) dst_apply_oz(dp, x, y, rows, rpr, sc, s, true);
  else if (dp.kind == 1) dct_inv_launch<double, double, double>(dp, x, y, rows, rpr, dp.ie, dp.io, sc, s, KC_DST64);
  else dst_apply_f64(dp, x, y, rows, rpr, sc, s);
}
void dst_inverse_f32_f2d(const DstPlan &dp, const float *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                         cudaStream_t s, bool rscale) {
  if (dp.kind == 1)
    dct_inv_launch<float, double, float>(dp, x, y, rows, rpr, dp.ie_f, dp.io_f, sc, s, KC_DST32_INV, rscale ? 2 : 0);
  else dst_apply_f32_f2d(dp, x, y, rows, rpr, sc, s, rscale);
}

void dst_apply_f64_simt(const DstPlan &dp, const double *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                        cudaStream_t s) {
  dst_simt_launch<double, double, double>(dp, x, y, rows, rpr, dp.su, dp.sv, sc, s, KC_DST64);
}
void dst_apply_f64(const DstPlan &dp, const double *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                   cudaStream_t s) {
  if (dp.oz) dst_apply_oz(dp, x, y, rows, rpr, sc, s);
  else dst_apply_f64_simt(dp, x, y, rows, rpr, sc, s);
}
void dst_apply_f32_d2f(const DstPlan &dp, const double *x, float *y, int rows, int rpr, const KrylovScalars *sc,
                       cudaStream_t s, bool rscale) {
  dst_simt_launch<double, float, float>(dp, x, y, rows, rpr, dp.su_f, dp.sv_f, sc, s, KC_DST32_FWD, rscale ? 1 : 0);
}
void dst_apply_f32_f2d(const DstPlan &dp, const float *x, double *y, int rows, int rpr, const KrylovScalars *sc,
                       cudaStream_t s, bool rscale) {
  dst_simt_launch<float, double, float>(dp, x, y, rows, rpr, dp.su_f, dp.sv_f, sc, s, KC_DST32_INV, rscale ? 2 : 0);
}

}  // namespace lag
