// Partitioned tridiagonal solve with precomputed factors (the preconditioner's z-direction step).
//
// Sec. 1 and Sec. 2.4 of the paper: after the transform along x, every x-mode j needs the solve of
// one tridiagonal system T_j along z, and T_j is the same for every right-hand side and every
// Krylov iteration and harmonic.  The paper uses the Dichotomy Algorithm: an O(N) preparatory
// step done once, then per right-hand side a partitioned elimination whose only exchange is an
// associative reduction over the partitions.  On GB300 the partitions are threads of one CTA:
//
//   rows are cut into P partitions of length L (rows >= nz are identity rows with zero data).
//   The first row of partitions 1..P-1 is a separator xi_p; the other rows form blocks I_p.
//   1. per block: g = T_I^{-1} d_I with the block's precomputed LU factors (fm = 1/pivot,
//      fc = c * fm, fa = sub-diagonal), forward then backward sweep;
//   2. the separators satisfy a (P-1)-unknown tridiagonal system whose matrix depends only on
//      T_j (precomputed) and whose right-hand side is d_sep - a g_{p-1}^last - c g_p^first;
//      one warp per mode solves it by parallel cyclic reduction in log2(P) shuffle levels
//      with precomputed per-level multipliers;
//   3. correction y_I = g - xi_p v - xi_{p+1} w with the precomputed spike vectors
//      v = T_I^{-1}(a_first e_first), w = T_I^{-1}(c_last e_last).
//
// The column tile of MT modes x all rows lives in shared memory: the right-hand side is read
// once and the solution written once (coalesced rows of MT consecutive modes).
#include <algorithm>

#include "internal.h"

namespace lag {

// ------------------------------------------------------------------------------ layout
bool tri_mode_tile_ok(int elem_bytes, int L, int mt) {
  if (elem_bytes == 4) return (mt == 8 || mt == 16 || (mt == 32 && L <= 32));
  return (mt == 4 || mt == 8);
}

void tri_choose_layout(TriFactors &tf, int elem_bytes, int want_P, int want_mt, bool general) {
  const int nz = tf.nz;
  int Pt = (want_P > 0) ? std::min(want_P, 32) : 32;
  while (Pt > 1 && nz / Pt < 2) Pt /= 2;  // at least 2 rows per partition
  // partition length: a power of two (the register kernel unrolls its sweeps over it)
  int L = 1;
  while (L * Pt < nz) L *= 2;
  if (Pt > 1 && L < 2) L = 2;
  // P = ceil(nz / L): only the last partition holds identity rows beyond nz, so every other
  // partition of a Toeplitz-in-z system shares the "first" or "middle" factor class
  int P = (nz + L - 1) / L;
  if (P <= 1) {
    P = 1;
    L = 1;
    while (L < nz) L *= 2;
  }
  tf.P = P;
  tf.L = L;
  tf.gen = general;
  tf.ncls = general ? P : 3;
  const int n = P - 1;
  int lev = 0;
  while ((1 << lev) < n) ++lev;
  tf.levels = lev;
  tf.nf = 3 + 3 * lev;
  const int nzp = P * L;
  auto threads = [&](int m) { return ((m * P + 31) / 32) * 32; };
  tf.reg = (L >= 2 && L <= 64 && (elem_bytes == 4 || L <= 32));
  if (tf.reg) {
    // register kernel: the mode tile (a compile-time constant of the kernel) sets the bytes a warp
    // reads per row and instruction: float32 8 / 16 / 32 modes (32 / 64 / 128 bytes, a warp covering
    // 4 / 2 / 1 partitions), float64 4 / 8 modes.  Default 16 (float32) and 4 (float64, bound by the
    // FP64 pipe rather than the loads); the autotuner times the others.
    int mt = (elem_bytes == 4) ? 16 : 4;
    if (want_mt > 0 && tri_mode_tile_ok(elem_bytes, L, want_mt)) mt = want_mt;
    tf.mt = mt;
    tf.threads = threads(mt);
    // constant coefficients: the 3 factor classes are staged in shared memory; general systems
    // (one factor set per partition) read theirs from global memory (L2)
    // + the reduced-system multipliers of the CTA's modes ([mt][nf][32]) when a CTA solves several
    // right-hand sides (read in the dependent PCR chain: shared memory instead of L2)
    tf.smem = (size_t)((general ? 0 : 5 * 3 * L * mt) + (3 * 32 + 33) * mt + mt * tf.nf * 32) * elem_bytes;
    return;
  }
  // shared-memory tile kernel: modes per CTA power of two <= 32, threads <= 1024,
  // tile <= ~104 KB (two CTAs per SM)
  const size_t budget = 104 * 1024;
  int mt = 32;
  while (mt > 1 && ((size_t)mt * nzp * elem_bytes > budget || threads(mt) > 1024)) mt /= 2;
  while (mt > 1 && mt / 2 >= tf.nx) mt /= 2;  // tiny grids: no idle half tiles
  tf.mt = mt;
  tf.threads = threads(mt);
  tf.smem = (size_t)nzp * mt * elem_bytes + (size_t)(3 * 32 + 33) * mt * elem_bytes;
  if (tf.smem > 200 * 1024)
    throw Error(LAG_EINVAL, "nz too large for the shared-memory column tile of the tridiagonal solve");
}

// ------------------------------------------------------------------------------ factors
// Matrix of mode j: sub a_k, diag b_k, super c_k (rows >= nz: identity).  Constant coefficients
// (Toeplitz in z): a = c = off, b = diag0 + ax lambda_j (+ top0 on row 0).  General coefficients
// (zf != null): a_k = -zf[k], c_k = -zf[k+1], b_k = zf[k] + zf[k+1] + zax[k] lambda_j + zd[k], with
// zf the face coefficients over dz^2 (layered: zf[0] = 0 under a free surface; cylindrical: the
// r-faces, zf[0] = 0 on the axis).  lambda_j: DST-I eigenvalues, or DCT-II ones for dct plans.
struct TriMatrix {
  double off, diag0, ax, dx2inv, nxp1;
  double top0;  // added to row 0's diagonal: off (= -az/dz^2) under a free surface, else 0
  const double *zf, *zax, *zd;
  int nz, perm_ku;
  int dct;  // modes of the DCT-II (zero-flux faces): lambda_j = 4/dx^2 sin^2(pi j / (2 nx))
  __device__ double sin2(int c) const {
    const int j = (perm_ku > 0) ? (c < perm_ku ? 2 * c : 2 * (c - perm_ku) + 1) : c;  // mode at column c
    const double s = dct ? sinpi((double)j / (2.0 * (nxp1 - 1.0))) : sinpi((double)(j + 1) / (2.0 * nxp1));
    return s * s;
  }
  // per-mode value handed to row(): the diagonal (constant) or lambda_j (layered)
  __device__ double mode_value(int c) const {
    if (zf != nullptr) return 4.0 * dx2inv * sin2(c);
    const int j = (perm_ku > 0) ? (c < perm_ku ? 2 * c : 2 * (c - perm_ku) + 1) : c;
    const double s = sinpi((double)(j + 1) / (2.0 * nxp1));
    return diag0 + ax * 4.0 * dx2inv * s * s;
  }
  __device__ void row(int k, double mv, double &a, double &b, double &c) const {
    if (k >= nz) { a = 0.0; b = 1.0; c = 0.0; return; }
    if (zf != nullptr) {
      a = (k >= 1) ? -zf[k] : 0.0;
      c = (k + 1 < nz) ? -zf[k + 1] : 0.0;
      b = zf[k] + zf[k + 1] + zax[k] * mv + zd[k];
      return;
    }
    a = (k >= 1) ? off : 0.0;
    b = (k == 0) ? mv + top0 : mv;
    c = (k + 1 < nz) ? off : 0.0;
  }
};

__device__ __forceinline__ int rep_partition(int cls, int P) { return cls == 0 ? 0 : (cls == 1 ? 1 : P - 1); }

// one thread per (mode j, factor set): block LU factors and spikes of one partition.  Constant
// coefficients: sets 0/1/2 are the representative first / middle / last partitions; general: set
// p is partition p.
__global__ void tri_factor_kernel(TriMatrix M, int nx, int P, int L, int gen, double *fm, double *fc,
                                  double *fa, double *sv, double *sw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int cls = blockIdx.y;
  if (j >= nx) return;
  const bool exists = gen || (cls == 0) || (cls == 1 && P >= 3) || (cls == 2 && P >= 2);
  const size_t base = (size_t)cls * L * nx + j;
  if (!exists) {
    for (int i = 0; i < L; ++i) {
      const size_t f = base + (size_t)i * nx;
      fm[f] = fc[f] = fa[f] = sv[f] = sw[f] = 0.0;
    }
    return;
  }
  const int p = gen ? cls : rep_partition(cls, P);
  const double mv = M.mode_value(j);
  const int i0 = (p == 0) ? 0 : 1;
  double a, b, c;
  // separator row slot (i = 0 of p >= 1) is unused by the sweeps
  if (i0 == 1) {
    const size_t f = base;
    fm[f] = fc[f] = fa[f] = sv[f] = sw[f] = 0.0;
  }
  double fc_prev = 0.0;
  for (int i = i0; i < L; ++i) {
    M.row(p * L + i, mv, a, b, c);
    const double den = (i == i0) ? b : b - a * fc_prev;
    const double m = 1.0 / den;
    const size_t f = base + (size_t)i * nx;
    fm[f] = m;
    fc[f] = c * m;
    fa[f] = (i == i0) ? 0.0 : a;
    fc_prev = c * m;
  }
  // spikes: v = T^{-1}(a_first e_first) (p >= 1), w = T^{-1}(c_last e_last) (p <= P-2)
  double a0, b0, c0, aL, bL, cL;
  M.row(p * L + i0, mv, a0, b0, c0);
  M.row(p * L + L - 1, mv, aL, bL, cL);
  const bool has_v = p >= 1, has_w = p <= P - 2;
  double vp = 0.0, wp = 0.0;
  for (int i = i0; i < L; ++i) {  // forward elimination of the two unit right-hand sides
    const size_t f = base + (size_t)i * nx;
    const double rv = (i == i0 && has_v) ? a0 : 0.0;
    const double rw = (i == L - 1 && has_w) ? cL : 0.0;
    vp = (i == i0) ? rv * fm[f] : (rv - fa[f] * vp) * fm[f];
    wp = (i == i0) ? rw * fm[f] : (rw - fa[f] * wp) * fm[f];
    sv[f] = vp;
    sw[f] = wp;
  }
  double vn = 0.0, wn = 0.0;
  for (int i = L - 1; i >= i0; --i) {  // back substitution
    const size_t f = base + (size_t)i * nx;
    const double v = (i == L - 1) ? sv[f] : sv[f] - fc[f] * vn;
    const double w = (i == L - 1) ? sw[f] : sw[f] - fc[f] * wn;
    sv[f] = v;
    sw[f] = w;
    vn = v;
    wn = w;
  }
}

// factor set of partition p: itself (general) or its class
__device__ __forceinline__ int set_of(int p, int P, int gen) { return gen ? p : (p == 0 ? 0 : (p == P - 1 ? 2 : 1)); }

// one thread per mode: reduced (separator) system and its PCR multipliers
__global__ void tri_reduced_kernel(TriMatrix M, int nx, int P, int L, int levels, int nf, int gen,
                                   const double *sv, const double *sw, double *red) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nx) return;
  const int n = P - 1;
  double A[32], B[32], C[32];
  double *R = red + (size_t)j * nf * 32;
  for (int f = 0; f < nf * 32; ++f) R[f] = 0.0;
  if (n <= 0) return;
  const double mv = M.mode_value(j);
  for (int q = 0; q < n; ++q) {
    const int p = q + 1;  // separator of partition p at row p L
    double a, b, c;
    M.row(p * L, mv, a, b, c);
    const size_t prevL = (size_t)set_of(p - 1, P, gen) * L * nx + (size_t)(L - 1) * nx + j;
    const size_t curF = (size_t)set_of(p, P, gen) * L * nx + (size_t)1 * nx + j;
    A[q] = -a * sv[prevL];
    B[q] = b - a * sw[prevL] - c * sv[curF];
    C[q] = -c * sw[curF];
    R[0 * 32 + q] = a;
    R[1 * 32 + q] = c;
  }
  // level-0 normalisation
  double ka[32], kc[32];
  for (int q = 0; q < n; ++q) {
    const double inv = 1.0 / B[q];
    R[2 * 32 + q] = inv;
    ka[q] = A[q] * inv;
    kc[q] = C[q] * inv;
  }
  for (int l = 0; l < levels; ++l) {
    const int s = 1 << l;
    double na[32], nc[32];
    for (int q = 0; q < n; ++q) {
      const double am = (q - s >= 0) ? ka[q - s] : 0.0, cm = (q - s >= 0) ? kc[q - s] : 0.0;
      const double ap = (q + s < n) ? ka[q + s] : 0.0, cp = (q + s < n) ? kc[q + s] : 0.0;
      const double den = 1.0 - ka[q] * cm - kc[q] * ap;
      const double inv = 1.0 / den;
      R[(3 + 3 * l) * 32 + q] = ka[q];
      R[(4 + 3 * l) * 32 + q] = kc[q];
      R[(5 + 3 * l) * 32 + q] = inv;
      na[q] = -ka[q] * am * inv;
      nc[q] = -kc[q] * cp * inv;
    }
    for (int q = 0; q < n; ++q) { ka[q] = na[q]; kc[q] = nc[q]; }
  }
}

void tri_build_factors(TriFactors &tf, DevBuf &store, const TriCoef &k, double dx, double dz, cudaStream_t s,
                       int perm_ku) {
  if (tf.gen != (k.zrows != nullptr)) throw Error(LAG_EINVAL, "factor layout does not match the coefficients");
  const size_t per = (size_t)tf.ncls * tf.L * tf.nx;
  const size_t nred = (size_t)tf.nx * tf.nf * 32;
  store.alloc(store.ctx, (5 * per + nred) * sizeof(double));
  double *base = store.as<double>();
  tf.fm = base;
  tf.fc = base + per;
  tf.fa = base + 2 * per;
  tf.sv = base + 3 * per;
  tf.sw = base + 4 * per;
  tf.red = base + 5 * per;
  TriMatrix M;
  M.off = -k.az / (dz * dz);
  M.diag0 = 2.0 * k.az / (dz * dz) + k.d;
  M.top0 = k.free_surface ? M.off : 0.0;
  M.ax = k.ax;
  M.dx2inv = 1.0 / (dx * dx);
  M.nxp1 = (double)(tf.nx + 1);
  M.zf = k.zrows;
  M.zax = k.zrows ? k.zrows + tf.nz + 1 : nullptr;
  M.zd = k.zrows ? k.zrows + 2 * tf.nz + 1 : nullptr;
  M.nz = tf.nz;
  M.perm_ku = perm_ku;
  M.dct = k.dct ? 1 : 0;
  if (k.dct && !k.zrows) throw Error(LAG_EINVAL, "DCT-II modes need general coefficients");
  const int gen = tf.gen ? 1 : 0;
  dim3 g1((tf.nx + 127) / 128, tf.ncls);
  tri_factor_kernel<<<g1, 128, 0, s>>>(M, tf.nx, tf.P, tf.L, gen, (double *)tf.fm, (double *)tf.fc,
                                       (double *)tf.fa, (double *)tf.sv, (double *)tf.sw);
  count_launch();
  LAG_LAUNCH_CHECK();
  tri_reduced_kernel<<<(tf.nx + 63) / 64, 64, 0, s>>>(M, tf.nx, tf.P, tf.L, tf.levels, tf.nf, gen,
                                                      (const double *)tf.sv, (const double *)tf.sw,
                                                      (double *)tf.red);
  count_launch();
  LAG_LAUNCH_CHECK();
}

__global__ void d2f_kernel(const double *a, float *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

void tri_make_f32(const TriFactors &t64, TriFactors &t32, DevBuf &store32, cudaStream_t s) {
  const size_t per = (size_t)t32.ncls * t32.L * t32.nx;
  const size_t nred = (size_t)t32.nx * t32.nf * 32;
  store32.alloc(store32.ctx, (5 * per + nred) * sizeof(float));
  float *base = store32.as<float>();
  t32.fm = base;
  t32.fc = base + per;
  t32.fa = base + 2 * per;
  t32.sv = base + 3 * per;
  t32.sw = base + 4 * per;
  t32.red = base + 5 * per;
  // the float64 set is contiguous in the same order
  d2f_kernel<<<1024, 256, 0, s>>>((const double *)t64.fm, base, 5 * per + nred);
  count_launch();
  LAG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------ solve
template <typename T>
__global__ void __launch_bounds__(1024) tri_solve_kernel(const T *__restrict__ din, T *__restrict__ yout,
                                                         int nz, int nx, int P, int L, int levels, int nf,
                                                         const T *__restrict__ fm, const T *__restrict__ fc,
                                                         const T *__restrict__ fa, const T *__restrict__ sv,
                                                         const T *__restrict__ sw, const T *__restrict__ red,
                                                         const KrylovScalars *__restrict__ sc, int pstride, int poff,
                                                         int ncomp, int mt, int gen) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *tile = reinterpret_cast<T *>(smem_raw);
  const int nzp = P * L;
  T *gF = tile + (size_t)nzp * mt;  // [mt][32]
  T *gL = gF + mt * 32;
  T *ds = gL + mt * 32;
  T *xi = ds + mt * 32;             // [mt][33]
  const int b = blockIdx.y * pstride + poff;  // plane index; right-hand side b / ncomp
  if (sc != nullptr && sc[b / ncomp].state != ST_RUN) return;
  const int j0 = blockIdx.x * mt;
  const int tid = threadIdx.x, nth = blockDim.x;
  const T *src = din + (size_t)b * nz * nx;
  T *dst = yout + (size_t)b * nz * nx;

  // 1. coalesced load of the [nz][mt] tile; identity rows beyond nz hold zero data
  for (int idx = tid; idx < nzp * mt; idx += nth) {
    const int r = idx / mt, c = idx - r * mt, j = j0 + c;
    tile[idx] = (r < nz && j < nx) ? src[(size_t)r * nx + j] : T(0);
  }
  __syncthreads();

  // 2. block-local sweeps: thread (c, p); threads beyond mt * P (warp padding) only synchronise
  const int c = tid % mt, p = tid / mt, j = j0 + c;
  const bool live = j < nx && p < P;
  const int i0 = (p == 0) ? 0 : 1;
  const size_t fb = (size_t)set_of(p, P, gen) * L * nx + j;
  T *col = tile + (size_t)p * L * mt + c;  // row i of this partition at col[i * mt]
  if (live) {
    T prev = T(0);
    for (int i = i0; i < L; ++i) {
      const size_t f = fb + (size_t)i * nx;
      T dv = col[i * mt];
      dv = (i == i0) ? dv * fm[f] : (dv - fa[f] * prev) * fm[f];
      col[i * mt] = dv;
      prev = dv;
    }
    T nxt = T(0);
    for (int i = L - 1; i >= i0; --i) {
      const size_t f = fb + (size_t)i * nx;
      const T g = (i == L - 1) ? col[i * mt] : col[i * mt] - fc[f] * nxt;
      col[i * mt] = g;
      nxt = g;
    }
    gF[c * 32 + p] = col[i0 * mt];
    gL[c * 32 + p] = col[(L - 1) * mt];
    ds[c * 32 + p] = (p >= 1) ? col[0] : T(0);
  }
  __syncthreads();

  // 3. separators: one warp per mode, lane q = separator of partition q + 1
  const int warp = tid >> 5, lane = tid & 31, nwarp = nth >> 5;  // nth is a multiple of 32
  const int n = P - 1;
  for (int cc = warp; n > 0 && cc < mt; cc += nwarp) {
    const int jj = j0 + cc;
    if (jj >= nx) continue;  // warp-uniform
    const T *R = red + (size_t)jj * nf * 32;
    const bool act = lane < n;
    T rq = T(0);
    if (act) {
      const int pp = lane + 1;
      rq = (ds[cc * 32 + pp] - R[lane] * gL[cc * 32 + pp - 1] - R[32 + lane] * gF[cc * 32 + pp]) * R[64 + lane];
    }
    for (int l = 0; l < levels; ++l) {
      const int s = 1 << l;
      T rm = __shfl_up_sync(0xffffffffu, rq, s);
      T rp = __shfl_down_sync(0xffffffffu, rq, s);
      if (lane < s) rm = T(0);
      if (lane + s >= n) rp = T(0);
      if (act) rq = (rq - R[(3 + 3 * l) * 32 + lane] * rm - R[(4 + 3 * l) * 32 + lane] * rp) * R[(5 + 3 * l) * 32 + lane];
    }
    xi[cc * 33 + lane + 1] = act ? rq : T(0);
    if (lane == 0) xi[cc * 33] = T(0);
  }
  __syncthreads();

  // 4. correction with the spike vectors
  if (n == 0 && tid < mt) xi[tid * 33] = T(0);
  __syncthreads();
  if (live) {
    const T xa = xi[c * 33 + p];
    const T xb = (p + 1 <= P - 1) ? xi[c * 33 + p + 1] : T(0);
    if (p >= 1) col[0] = xa;
    for (int i = i0; i < L; ++i) {
      const size_t f = fb + (size_t)i * nx;
      col[i * mt] = col[i * mt] - xa * sv[f] - xb * sw[f];
    }
  }
  __syncthreads();

  // 5. coalesced store
  for (int idx = tid; idx < nz * mt; idx += nth) {
    const int r = idx / mt, cc = idx - r * mt, jj = j0 + cc;
    if (jj < nx) dst[(size_t)r * nx + jj] = tile[idx];
  }
}


// Register-resident variant (partition length L a compile-time power of two): thread (c, p) keeps
// the L values of its partition in registers, loaded straight from global memory (a warp reads
// rows of MT consecutive modes: whole 32-byte sectors, 64 bytes per row for float32) and stored
// back the same way; only the separator ends and the separator solution pass through shared
// memory.  Constant coefficients (GEN false): the factors of the CTA's modes (3 classes x L rows)
// are staged once in shared memory and reused for the `per_cta` right-hand sides the CTA solves in
// turn.  General systems (GEN true, one factor set per partition): each thread reads its
// partition's factors from global memory with the same access pattern as the data (L2-resident
// across the right-hand sides of the CTA).
// occupancy target of the register kernel: 64 (float32) / 128 (float64) registers a thread at
// L <= 32, twice that at L = 64; general systems (factor addresses per row) twice that again at
// L >= 32
template <typename T, int L, int MT, bool GEN>
struct RegBounds {
  static constexpr int threads = MT * 32;
  static constexpr int per_sm = (sizeof(T) == 8 ? 512 : 1024) / (L >= 64 ? 2 : 1) / ((GEN && L >= 32) ? 2 : 1);
  static constexpr int blocks = per_sm / threads > 0 ? per_sm / threads : 1;
};

// RZ (float64, one component, din != yout): also the dot (d, y) of each plane, summed over the CTAs
// of its modes (block sums published into rz, the last CTA combining them in CTA order), and PCG's
// beta from it into scw (see tri_solve_f64_rz)
template <typename T, int L, int MT, bool GEN, bool RZ>
__global__ void __launch_bounds__(RegBounds<T, L, MT, GEN>::threads, RegBounds<T, L, MT, GEN>::blocks) tri_solve_reg_kernel(const T *__restrict__ din, T *__restrict__ yout, int nz,
                                                               int nx, int P, int levels, int nf,
                                                               const T *__restrict__ fm, const T *__restrict__ fc,
                                                               const T *__restrict__ fa, const T *__restrict__ sv,
                                                               const T *__restrict__ sw, const T *__restrict__ red,
                                                               const KrylovScalars *__restrict__ sc, int pstride,
                                                               int poff, int ncomp, int nplanes, int per_cta,
                                                               KrylovScalars *scw, Reduce rz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NCR = GEN ? 0 : 3 * L;       // staged factor rows: 3 classes x L
  T *F = reinterpret_cast<T *>(smem_raw);    // [5][NCR][MT]: fm, fa, fc, sv, sw
  T *gF = F + 5 * NCR * MT;                  // [MT][32]
  T *gL = gF + MT * 32;
  T *ds = gL + MT * 32;
  T *xi = ds + MT * 32;                      // [MT][33]
  T *Rs = xi + MT * 33;                      // [MT][nf][32]: reduced systems of the CTA's modes
  const int j0 = blockIdx.x * MT;
  const int tid = threadIdx.x, nth = blockDim.x;
  const bool stage_red = per_cta > 1;        // staging pays off over several right-hand sides
  if (stage_red)
    for (int idx = tid; idx < MT * nf * 32; idx += nth)  // one contiguous block of red
      Rs[idx] = (j0 + idx / (nf * 32) < nx) ? red[(size_t)j0 * nf * 32 + idx] : T(0);
  // stage the factors of this CTA's modes: row-major [row][MT], MT a power of two
  if constexpr (!GEN) {
    const int cm = tid % MT, r0 = tid / MT, rstep = nth / MT;
    const int j = j0 + cm;
    for (int row = r0; row < NCR; row += rstep) {
      const size_t g = (size_t)row * nx + j;
      const bool ok = j < nx;
      F[(0 * NCR + row) * MT + cm] = ok ? fm[g] : T(0);
      F[(1 * NCR + row) * MT + cm] = ok ? fa[g] : T(0);
      F[(2 * NCR + row) * MT + cm] = ok ? fc[g] : T(0);
      F[(3 * NCR + row) * MT + cm] = ok ? sv[g] : T(0);
      F[(4 * NCR + row) * MT + cm] = ok ? sw[g] : T(0);
    }
  }
  const int c = tid % MT, p = tid / MT, j = j0 + c;
  const bool col_ok = j < nx && p < P;
  const int i0 = (p == 0) ? 0 : 1;
  // factor rows of this thread's partition: stride FS between rows
  constexpr int FS_SMEM = MT;
  const int FS = GEN ? nx : FS_SMEM;
  const size_t fo = GEN ? (size_t)p * L * nx + j : (size_t)(set_of(p, P, 0) * L) * MT + c;
  const T *Fm = (GEN ? fm : F + 0 * NCR * MT) + fo;
  const T *Fa = (GEN ? fa : F + 1 * NCR * MT) + fo;
  const T *Fc = (GEN ? fc : F + 2 * NCR * MT) + fo;
  const T *Sv = (GEN ? sv : F + 3 * NCR * MT) + fo;
  const T *Sw = (GEN ? sw : F + 4 * NCR * MT) + fo;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nth >> 5;
  const int n = P - 1;
  __syncthreads();
  for (int k = 0; k < per_cta; ++k) {
    const int bi = blockIdx.y * per_cta + k;
    if (bi >= nplanes) break;                                  // uniform over the CTA
    const int b = bi * pstride + poff;
    if (sc != nullptr && sc[b / ncomp].state != ST_RUN) continue;  // uniform over the CTA
    const bool live = col_ok;
    const T *src = din + (size_t)b * nz * nx + j;
    T *dst = yout + (size_t)b * nz * nx + j;
    T v[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const int r = p * L + i;
      v[i] = (live && r < nz) ? src[(size_t)r * nx] : T(0);
    }
    const T dsep = v[0];  // separator row value (p >= 1)
    if (live) {
      // forward elimination over the block rows i0..L-1, then back substitution: v = T_I^{-1} d_I
      T prev = T(0);
#pragma unroll
      for (int i = 0; i < L; ++i) {
        if (i < i0) continue;
        const T m = Fm[i * FS];
        v[i] = (i == i0) ? v[i] * m : (v[i] - Fa[i * FS] * prev) * m;
        prev = v[i];
      }
#pragma unroll
      for (int i = L - 2; i >= 0; --i) {
        if (i < i0) continue;
        v[i] = v[i] - Fc[i * FS] * v[i + 1];
      }
      gF[c * 32 + p] = (i0 == 0) ? v[0] : v[1];
      gL[c * 32 + p] = v[L - 1];
      ds[c * 32 + p] = (p >= 1) ? dsep : T(0);
    }
    __syncthreads();
    // separators: one warp per mode, parallel cyclic reduction in shuffles (precomputed multipliers)
    for (int cc = warp; n > 0 && cc < MT; cc += nwarp) {
      const int jj = j0 + cc;
      if (jj >= nx) continue;  // warp-uniform
      const T *R = stage_red ? Rs + (size_t)cc * nf * 32 : red + (size_t)jj * nf * 32;
      const bool act = lane < n;
      T rq = T(0);
      if (act) {
        const int pp = lane + 1;
        rq = (ds[cc * 32 + pp] - R[lane] * gL[cc * 32 + pp - 1] - R[32 + lane] * gF[cc * 32 + pp]) * R[64 + lane];
      }
      for (int l = 0; l < levels; ++l) {
        const int s = 1 << l;
        T rm = __shfl_up_sync(0xffffffffu, rq, s);
        T rp = __shfl_down_sync(0xffffffffu, rq, s);
        if (lane < s) rm = T(0);
        if (lane + s >= n) rp = T(0);
        if (act) rq = (rq - R[(3 + 3 * l) * 32 + lane] * rm - R[(4 + 3 * l) * 32 + lane] * rp) * R[(5 + 3 * l) * 32 + lane];
      }
      xi[cc * 33 + lane + 1] = act ? rq : T(0);
      if (lane == 0) xi[cc * 33] = T(0);
    }
    if (n == 0 && tid < MT) xi[tid * 33] = T(0);
    __syncthreads();
    T dot = T(0);
    if (live) {
      // correction with the spike vectors, store
      const T xa = xi[c * 33 + p];
      const T xb = (p + 1 <= P - 1) ? xi[c * 33 + p + 1] : T(0);
#pragma unroll
      for (int i = 0; i < L; ++i) {
        const int r = p * L + i;
        const T y = (i < i0) ? xa : v[i] - xa * Sv[i * FS] - xb * Sw[i * FS];
        if (r < nz) {
          dst[(size_t)r * nx] = y;
          if constexpr (RZ) dot = fma(src[(size_t)r * nx], y, dot);  // d is still intact (din != yout)
        }
      }
    }
    if constexpr (RZ) {
      double v1[1] = {(double)dot}, tot[1];
      __shared__ double rsh[32];
      block_sum<1>(v1, rsh);
      if (publish_partials<1>(rz, b, blockIdx.x, gridDim.x, v1, tot)) {
        KrylovScalars &S = scw[b];
        const double rz_new = tot[0];
        S.beta = (S.iters == 0) ? 0.0 : rz_new / S.rz;
        S.rz = rz_new;
        if (!isfinite(S.beta) || !isfinite(rz_new)) S.state = ST_NAN;
      }
    }
    __syncthreads();  // gF/gL/ds/xi are reused by the next right-hand side
  }
}

// the optional (d, y) dot of a float64 solve: scalars to update and the reduction to sum into
struct TriRz {
  KrylovScalars *sc;
  Reduce red;
};

template <typename T, int L, int MT, bool GEN, bool RZ>
static void tri_reg_launch_rz(const TriFactors &tf, const T *d, T *y, int nrhs, const KrylovScalars *sc,
                              cudaStream_t s, int pstride, int poff, int ncomp, const TriRz *rz) {
  static PerDeviceOnce attr_done;
  attr_done.run([] {
    LAG_CUDA_CHECK(cudaFuncSetAttribute(tri_solve_reg_kernel<T, L, MT, GEN, RZ>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  // several right-hand sides per CTA when there are plenty of CTAs anyway (factor reuse)
  const int ctas_x = (tf.nx + MT - 1) / MT;
  int per_cta = 1;
  while (per_cta < 8 && (long long)ctas_x * ((nrhs + 2 * per_cta - 1) / (2 * per_cta)) >= 152 * 8) per_cta *= 2;
  dim3 grid(ctas_x, (nrhs + per_cta - 1) / per_cta);
  tri_solve_reg_kernel<T, L, MT, GEN, RZ><<<grid, tf.threads, tf.smem, s>>>(
      d, y, tf.nz, tf.nx, tf.P, tf.levels, tf.nf, (const T *)tf.fm, (const T *)tf.fc, (const T *)tf.fa,
      (const T *)tf.sv, (const T *)tf.sw, (const T *)tf.red, sc, pstride, poff, ncomp, nrhs, per_cta,
      rz != nullptr ? rz->sc : nullptr, rz != nullptr ? rz->red : Reduce{});
}

template <typename T, int L, int MT, bool GEN>
static void tri_reg_launch_mt(const TriFactors &tf, const T *d, T *y, int nrhs, const KrylovScalars *sc,
                              cudaStream_t s, int pstride, int poff, int ncomp, const TriRz *rz) {
  if constexpr (sizeof(T) == 8) {
    if (rz != nullptr) {
      tri_reg_launch_rz<T, L, MT, GEN, true>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
      return;
    }
  }
  tri_reg_launch_rz<T, L, MT, GEN, false>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, nullptr);
}

template <typename T, int L, int MT>
static void tri_reg_launch_gen(const TriFactors &tf, const T *d, T *y, int nrhs, const KrylovScalars *sc,
                               cudaStream_t s, int pstride, int poff, int ncomp, const TriRz *rz) {
  if (tf.gen) tri_reg_launch_mt<T, L, MT, true>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
  else tri_reg_launch_mt<T, L, MT, false>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
}

template <typename T, int L>
static void tri_reg_launch(const TriFactors &tf, const T *d, T *y, int nrhs, const KrylovScalars *sc, cudaStream_t s,
                           int pstride, int poff, int ncomp, const TriRz *rz) {
  if constexpr (sizeof(T) == 4) {
    if (tf.mt == 8) tri_reg_launch_gen<T, L, 8>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
    else if constexpr (L <= 32) {
      if (tf.mt == 32) tri_reg_launch_gen<T, L, 32>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
      else tri_reg_launch_gen<T, L, 16>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
    } else {
      tri_reg_launch_gen<T, L, 16>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
    }
  } else {
    if (tf.mt == 8) tri_reg_launch_gen<T, L, 8>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
    else tri_reg_launch_gen<T, L, 4>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz);
  }
}

template <typename T>
static void tri_launch(const TriFactors &tf, const T *d, T *y, int nrhs, const KrylovScalars *sc,
                       cudaStream_t s, int pstride, int poff, int ncomp, const TriRz *rz = nullptr) {
  if (nrhs <= 0) return;
  static PerDeviceOnce attr_done;
  attr_done.run([] {
    LAG_CUDA_CHECK(cudaFuncSetAttribute(tri_solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  ProfScope prof(sizeof(T) == 8 ? KC_TRI64 : KC_TRI32, s);
  if (tf.reg) {
    switch (tf.L) {
      case 2: tri_reg_launch<T, 2>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz); break;
      case 4: tri_reg_launch<T, 4>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz); break;
      case 8: tri_reg_launch<T, 8>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz); break;
      case 16: tri_reg_launch<T, 16>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz); break;
      case 32: tri_reg_launch<T, 32>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz); break;
      default: tri_reg_launch<T, 64>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp, rz); break;
    }
    count_launch();
    LAG_LAUNCH_CHECK();
    return;
  }
  if (rz != nullptr) throw Error(LAG_EINVAL, "the (d, y) dot needs the register tridiagonal kernel");
  dim3 grid((tf.nx + tf.mt - 1) / tf.mt, nrhs);
  tri_solve_kernel<T><<<grid, tf.threads, tf.smem, s>>>(
      d, y, tf.nz, tf.nx, tf.P, tf.L, tf.levels, tf.nf, (const T *)tf.fm, (const T *)tf.fc,
      (const T *)tf.fa, (const T *)tf.sv, (const T *)tf.sw, (const T *)tf.red, sc, pstride, poff, ncomp, tf.mt,
      tf.gen ? 1 : 0);
  count_launch();
  LAG_LAUNCH_CHECK();
}

void tri_solve_f64(const TriFactors &tf, const double *d, double *y, int nrhs, const KrylovScalars *sc,
                   cudaStream_t s, int pstride, int poff, int ncomp) {
  tri_launch<double>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp);
}
void tri_solve_f32(const TriFactors &tf, const float *d, float *y, int nrhs, const KrylovScalars *sc,
                   cudaStream_t s, int pstride, int poff, int ncomp) {
  tri_launch<float>(tf, d, y, nrhs, sc, s, pstride, poff, ncomp);
}

bool tri_rz_fusable(const TriFactors &tf, const Reduce &red) {
  return tf.reg && tf.mt > 0 && (tf.nx + tf.mt - 1) / tf.mt <= red.nblk;
}
void tri_solve_f64_rz(const TriFactors &tf, const double *d, double *y, int nrhs, KrylovScalars *sc,
                      const Reduce &red, cudaStream_t s) {
  if (d == y) throw Error(LAG_EINVAL, "tri_solve_f64_rz: d and y must differ");
  if (!tri_rz_fusable(tf, red)) throw Error(LAG_EINVAL, "tri_solve_f64_rz: not available for this plan");
  const TriRz rz{sc, red};
  tri_launch<double>(tf, d, y, nrhs, sc, s, 1, 0, 1, &rz);
}

}  // namespace lag
