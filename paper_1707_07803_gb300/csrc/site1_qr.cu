// Site-1 QR of Algs. 5.2/5.3 (A1^T = Q~ R~, the (I1 t) x K matrix Y of the site-1 core) by
// CholeskyQR2 in ONE cooperative launch with three grid barriers.
//
// Nothing in a pass is serialised on one CTA:
//   * the Gram G = Y^T Y is computed by column tiles: CTA b takes 4 x 4 tiles of the upper
//     triangle and sums each entry over all rows (read from L2), so G is written once, with no
//     partial Grams and no reduction step; the summation order is fixed (deterministic);
//   * after a grid barrier every CTA reads G and factors it itself: the K-step Cholesky chain is
//     the same on every SM (identical inputs, identical code: identical factors), so no factor
//     travels back through L2 and no barrier waits for one CTA;
//   * every CTA then applies the factor to its own rows (spread over the whole grid).
// Pass 1 factors G1 in the square-root-free form G1 = U^T D U; it only has to precondition, since
// Y = Q1 R1 holds exactly for the R1 the solve uses. Pass 2 sees G2 = Q1^T Q1 = I + E with
// |E| ~ cond(Y)^2 eps. When G2 is not within 0.5 / K of the identity (outside the regime in which
// CholeskyQR2 is orthogonal to rounding level) *flag is set and the caller falls back to
// Householder with the core unchanged. When K max|E| <= 1e-4 its factor is taken from the series
// of the Cholesky factor of I + E instead of a K-step pivot chain: with Phi(M) = triu(M) -
// diag(M) / 2 (so that Phi(M) + Phi(M)^T = M for symmetric M), R2 = I + X solves X + X^T + X^T X
// = E exactly when X = Phi(E - X^T X); three fixed-point steps from X = 0 leave R2^T R2 - G2 =
// O(|E|^4) <= (K max|E|)^4 <= 1e-16, below rounding. Otherwise G2 is factored like G1. The
// result is R = R2 R1 and Q = Y R1^{-1} R2^{-1}.
#include <algorithm>

#include "dev_common.cuh"
#include "grid_sync.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

constexpr int kS1Threads = 256;
constexpr int kS1MaxK = 32;
constexpr int kS1MaxRowsPerCta = 384;
constexpr int kS1Ld = kS1MaxK + 1;  // leading dimension of the K x K work matrices (no bank conflicts)
constexpr int kS1Tile = 4;          // Gram tiles of 4 x 4 column pairs
constexpr int kS1Chunk = 512;       // rows of a tile's two column blocks staged per step

struct Site1Args {
  double *core0;          // (1, I1, K, t)
  const int64_t *t_dev;   // t in device memory (rank left there by the rounding), or null
  int I1, K, t;           // t: the rank when t_dev is null, else its upper bound
  int core_out;           // write Q~ back into core0's layout instead of Qout
  const int *gate;        // when not null and 0 on the device: do nothing (an earlier step declined)
  double *Q1;           // m x K scratch, column-major (ld m): the first pass's Q for the second Gram
  double *G;            // K x K scratch: the current pass's Gram (column-major, symmetric)
  double *Rout;         // K x K: R = R2 R1 (column-major, upper)
  double *Qout;         // m x K, column-major
  int *flag;            // set when the factorisation cannot be trusted
  unsigned *bar;
  int *status;
};

// Element (row, c) of the site-1 matrix: core (row mod I1, c, row div I1).
__device__ __forceinline__ int64_t ycore(int row, int c, int I1, int K) {
  return (int64_t)(row % I1) + (int64_t)I1 * (c + (int64_t)K * (row / I1));
}

struct CoreAt {  // Y read from the core (written by earlier launches)
  const double *core;
  int I1, K;
  __device__ double operator()(int r, int c) const { return core[ycore(r, c, I1, K)]; }
};

struct ColAt {  // column-major m x K matrix written by other CTAs of this launch (through L2)
  const double *x;
  int m;
  __device__ double operator()(int r, int c) const { return __ldcg(x + r + (int64_t)m * c); }
};

// Pass-1 pivot reciprocal: the FP64 approximate reciprocal instruction refined by one Newton step
// (its error is far below what preconditioning needs: Y = Q1 R1 holds for the R1 applied).
__device__ __forceinline__ double rcp_precondition(double x) {
  double q;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(q) : "d"(x));
  return fma(q, fma(-x, q, 1.0), q);
}

// G (K x K, global) <- X^T X for the m x K matrix X (element (r, c) = x_at(r, c)): CTA b takes
// tiles b, b + gridDim.x, ... of the 4 x 4-tiled upper triangle; a tile's two column blocks are
// staged in shared memory kS1Chunk rows at a time, thread (pair, slice) sums rows slice, slice +
// 16, ..., and the 16 slices of a pair are added in order. cols: 2 kS1Tile kS1Chunk doubles.
template <typename XAt>
__device__ void gram_tiles(int m, int K, const XAt &x_at, double *G, double *cols) {
  __shared__ double red[16][17];
  const int nt = (K + kS1Tile - 1) / kS1Tile, ntiles = nt * (nt + 1) / 2;
  const int pr = threadIdx.x & 15, sl = threadIdx.x >> 4;
  const int pi = pr & 3, pj = pr >> 2;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int bi = 0, rem = tile;  // tile -> (bi, bj), bi <= bj, row by row over the upper triangle
    while (rem >= nt - bi) {
      rem -= nt - bi;
      ++bi;
    }
    const int bj = bi + rem;
    const int ci = bi * kS1Tile + pi, cj = bj * kS1Tile + pj;
    double acc = 0.0;
    for (int r0 = 0; r0 < m; r0 += kS1Chunk) {
      const int nr = min(kS1Chunk, m - r0);
      for (int x = threadIdx.x; x < 2 * kS1Tile * nr; x += blockDim.x) {
        const int q = x / nr, rr = x - q * nr;  // column slot q: 0..3 block bi, 4..7 block bj
        const int c = q < kS1Tile ? bi * kS1Tile + q : bj * kS1Tile + q - kS1Tile;
        cols[q * kS1Chunk + rr] = c < K ? x_at(r0 + rr, c) : 0.0;
      }
      __syncthreads();
      const double *xa = cols + pi * kS1Chunk, *xb = cols + (kS1Tile + pj) * kS1Chunk;
      for (int rr = sl; rr < nr; rr += 16) acc = fma(xa[rr], xb[rr], acc);
      __syncthreads();
    }
    red[pr][sl] = acc;
    __syncthreads();
    if (threadIdx.x < 16 && ci < K && cj < K) {
      double s = 0.0;
      for (int q = 0; q < 16; ++q) s += red[pr][q];
      G[ci + K * cj] = s;
      if (bi != bj) G[cj + K * ci] = s;
    }
    __syncthreads();
  }
}

// Square-root-free Cholesky G = U^T D U of the K x K matrix a (shared, column-major with leading
// dimension kS1Ld, K <= 32) on one CTA: on return a(i, l) = d_i u_il for i <= l, dinv[i] = 1 / d_i. Thread (lane, warp)
// owns the elements (i = lane, l = warp + 8 u). The owner of the next diagonal element forms
// its reciprocal right after its own update, so it overlaps the other updates of the step.
// precond: pass-1 reciprocals (rcp_precondition), else full FP64 ones. Returns false (uniform
// over the CTA) when a pivot is not positive and finite.
__device__ bool cta_ldl(double *a, int K, double *dinv, bool precond) {
  __shared__ int s_bad;
  const int i = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kW = kS1Threads / 32;
  if (threadIdx.x == 0) {
    const double d0 = a[0];
    s_bad = !(d0 > 0.0) || !isfinite(d0);
    if (!s_bad) dinv[0] = precond ? rcp_precondition(d0) : rcp_f64(d0);
  }
  __syncthreads();
  if (s_bad) return false;
  const bool own_diag = i < K && (i % kW) == w;  // this thread holds (i, i)
  for (int j = 0; j < K; ++j) {
    if (i > j && i < K) {
      const double f = a[j + kS1Ld * i] * dinv[j];
      if (own_diag && i == j + 1) {
        const double v = fma(-f, a[j + kS1Ld * i], a[i + kS1Ld * i]);
        a[i + kS1Ld * i] = v;
        if (!(v > 0.0) || !isfinite(v))
          s_bad = 1;
        else
          dinv[j + 1] = precond ? rcp_precondition(v) : rcp_f64(v);
      }
      for (int l = w; l < K; l += kW) {
        if (l < i || (l == i && i == j + 1)) continue;
        a[i + kS1Ld * l] = fma(-f, a[j + kS1Ld * l], a[i + kS1Ld * l]);
      }
    }
    __syncthreads();
    if (s_bad) return false;
  }
  return true;
}

// y <- y R^{-1} for the rows of ys (row-major, leading dimension K + 1), warp per row, lane c
// owns column c. R is given as Ru (upper, leading dimension kS1Ld) with u_jc = Ru(j, c) sc_j the
// unit upper factor of R = diag(R_jj) U and fin_c = 1 / R_cc: step j broadcasts the current y_j
// and lanes c > j subtract y_j u_jc; finally x_c = y_c fin_c. (Square-root-free factor: Ru = D U,
// sc = 1 / d, fin = 1 / sqrt(d); explicit R: Ru = R, sc = fin = 1 / diag(R).)
__device__ void rows_solve(double *ys, int nr, int K, const double *Ru, const double *sc, const double *fin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, ld = K + 1;
  double u[kS1MaxK];
#pragma unroll
  for (int j = 0; j < kS1MaxK; ++j) u[j] = (lane < K && j < lane) ? Ru[j + kS1Ld * lane] * sc[j] : 0.0;
  const double rd = lane < K ? fin[lane] : 0.0;
  for (int rr = warp; rr < nr; rr += nw) {
    double y = lane < K ? ys[rr * ld + lane] : 0.0;
#pragma unroll
    for (int j = 0; j < kS1MaxK; ++j) {
      if (j >= K) break;
      const double yj = __shfl_sync(0xffffffffu, y, j);
      y = fma(-yj, u[j], y);  // u[j] = 0 for j >= lane
    }
    if (lane < K) ys[rr * ld + lane] = y * rd;
  }
}

// X <- Phi(E - X^T X) for E = a - I (a: G2 in shared memory), the fixed-point step of the series
// of the Cholesky factor of I + E; xs, ps: K x K work (leading dimension kS1Ld), xs = X on entry
// (ignored when first) and on exit. (X^T X)(i, l) = sum_{q <= i} X(q, i) X(q, l) for i <= l (X is
// upper triangular): the packed upper triangle is spread over the whole CTA, one entry per thread
// and pass, summed in four interleaved chains; only the upper triangle of ps is read. With f32 the
// sums run on the FP32 pipe from xs32, an FP32 copy of X kept beside it: X^T X is a correction of
// size ~K emax^2 (emax = max |E|), so its FP32 rounding error is at most ~K^2 2^-24 emax^2, below
// 1e-17 when K emax <= 1e-5 (the caller's condition for f32); on GB300 the FP64 pipe issues one
// warp instruction per ~64 cycles, so the FP64 sums cost ~5 us per step and the FP32 ones ~0.3.
__device__ void chol_series_step(const double *a, double *xs, float *xs32, double *ps, int K, bool first, bool f32) {
  if (!first) {
    const int E = K * (K + 1) / 2;
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) {
      int i, l;
      packed_upper(idx, false, i, l);  // i <= l
      double sum;
      int q = 0;
      if (f32) {
        const float *xi = xs32 + kS1Ld * i, *xl = xs32 + kS1Ld * l;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        for (; q + 3 <= i; q += 4) {
          s0 = fmaf(xi[q], xl[q], s0);
          s1 = fmaf(xi[q + 1], xl[q + 1], s1);
          s2 = fmaf(xi[q + 2], xl[q + 2], s2);
          s3 = fmaf(xi[q + 3], xl[q + 3], s3);
        }
        for (; q <= i; ++q) s0 = fmaf(xi[q], xl[q], s0);
        sum = (double)((s0 + s1) + (s2 + s3));
      } else {
        const double *xi = xs + kS1Ld * i, *xl = xs + kS1Ld * l;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (; q + 3 <= i; q += 4) {
          s0 = fma(xi[q], xl[q], s0);
          s1 = fma(xi[q + 1], xl[q + 1], s1);
          s2 = fma(xi[q + 2], xl[q + 2], s2);
          s3 = fma(xi[q + 3], xl[q + 3], s3);
        }
        for (; q <= i; ++q) s0 = fma(xi[q], xl[q], s0);
        sum = (s0 + s1) + (s2 + s3);
      }
      ps[i + kS1Ld * l] = sum;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e % K, l = e / K;
    const double m = a[i + kS1Ld * l] - (i == l ? 1.0 : 0.0) - (first || i > l ? 0.0 : ps[i + kS1Ld * l]);
    const double x = i < l ? m : (i == l ? 0.5 * m : 0.0);
    xs[i + kS1Ld * l] = x;
    if (f32) xs32[i + kS1Ld * l] = (float)x;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kS1Threads) k_site1_cholqr2(Site1Args a) {
  unsigned epoch = 0;  // grid barriers passed by this CTA
  extern __shared__ double dyn[];         // own rows (leading dimension K + 1), then tile staging
  __shared__ double am[kS1MaxK * kS1Ld];   // the current Gram, then its factor
  __shared__ double r1s[kS1MaxK * kS1Ld];  // R1
  __shared__ double xs[kS1MaxK * kS1Ld];   // R2 (series: X, then I + X)
  __shared__ double ps[kS1MaxK * kS1Ld];   // series work
  __shared__ float xs32[kS1MaxK * kS1Ld];  // series: an FP32 copy of X
  __shared__ double dinv[kS1MaxK], rd1[kS1MaxK], rd2[kS1MaxK], rdq[kS1MaxK];
  __shared__ unsigned long long s_emax;
  if (a.gate && __ldcg(a.gate) == 0) return;  // uniform: written by an earlier launch
  const int K = a.K, I1 = a.I1, tid = threadIdx.x, nthr = blockDim.x;
  const int64_t td = a.t_dev ? __ldcg(a.t_dev) : a.t;
  if (td < 1 || td > a.t) {  // outside the bound the launch was sized for: leave it to the fallback
    if (blockIdx.x == 0 && tid == 0) *a.flag = 1;
    return;
  }
  const int m = I1 * (int)td;
  const int ld = K + 1;
  const int rpc = (m + (int)gridDim.x - 1) / (int)gridDim.x;  // rows per CTA (the host sized for the bound)
  const int r0 = blockIdx.x * rpc;
  const int nr = max(0, min(rpc, m - r0));
  double *ys = dyn, *cols = dyn + (size_t)rpc * ld;
  if (blockIdx.x == 0 && tid == 0) *a.flag = 0;
  // own rows of Y: row i + I1 r, column c <- core (i, c, r)
  for (int x = tid; x < nr * K; x += nthr) {
    const int rr = x % nr, c = x / nr;
    ys[rr * ld + c] = a.core0[ycore(r0 + rr, c, I1, K)];
  }
  // ---- pass 1: G1 = Y^T Y by tiles, then every CTA factors it and solves its rows
  gram_tiles(m, K, CoreAt{a.core0, I1, K}, a.G, cols);
  grid_barrier(a.bar, a.status, epoch);
  for (int e = tid; e < K * K; e += nthr) am[(e % K) + kS1Ld * (e / K)] = __ldcg(a.G + e);
  __syncthreads();
  if (!cta_ldl(am, K, dinv, true)) {
    if (blockIdx.x == 0 && tid == 0) *a.flag = 1;
    return;  // uniform: every CTA factored the same matrix
  }
  // the solve scales row j of D U by rd1_j^2 = 1 / d_j to rounding (not by the preconditioning
  // reciprocal dinv_j), so Y = Q1 R1 holds to rounding for the R1 = D^{1/2} U kept for R = R2 R1
  if (tid < K) {
    rd1[tid] = rsqrt_f64(am[tid + kS1Ld * tid]);
    rdq[tid] = rd1[tid] * rd1[tid];
  }
  __syncthreads();
  for (int e = tid; e < K * K; e += nthr) {  // R1(i, l) = d_i u_il / sqrt(d_i)
    const int i = e % K, l = e / K;
    r1s[i + kS1Ld * l] = i <= l ? am[i + kS1Ld * l] * rd1[i] : 0.0;
  }
  rows_solve(ys, nr, K, am, rdq, rd1);
  __syncthreads();
  for (int x = tid; x < nr * K; x += nthr) {  // Q1 rows for the second Gram
    const int rr = x % nr, c = x / nr;
    a.Q1[(r0 + rr) + (int64_t)m * c] = ys[rr * ld + c];
  }
  grid_barrier(a.bar, a.status, epoch);
  // ---- pass 2: G2 = Q1^T Q1 by tiles, checked and factored by every CTA
  gram_tiles(m, K, ColAt{a.Q1, m}, a.G, cols);
  grid_barrier(a.bar, a.status, epoch);
  if (tid == 0) s_emax = 0ull;
  double dev = 0.0;
  for (int e = tid; e < K * K; e += nthr) {
    const int i = e % K, l = e / K;
    const double g = __ldcg(a.G + e);
    am[i + kS1Ld * l] = g;
    const double d = fabs(g - (i == l ? 1.0 : 0.0));
    dev = (d > dev || d != d) ? d : dev;  // a NaN wins (and fails the checks below)
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_xor_sync(0xffffffffu, dev, o);
    dev = (x > dev || x != x) ? x : dev;
  }
  __syncthreads();
  // non-negative doubles order like their bit patterns (a NaN's is larger than any)
  if ((tid & 31) == 0) atomicMax(&s_emax, (unsigned long long)__double_as_longlong(dev));
  __syncthreads();
  const double emax = __longlong_as_double((long long)s_emax);
  if (!(emax <= 0.5 / K)) {
    if (blockIdx.x == 0 && tid == 0) *a.flag = 1;
    return;  // uniform; the core is unchanged
  }
  if (K * emax <= 1e-4) {  // R2 = I + X from three steps of the series
    const bool f32 = K * emax <= 1e-5;  // uniform: every CTA read the same Gram
    chol_series_step(am, xs, xs32, ps, K, true, f32);
    chol_series_step(am, xs, xs32, ps, K, false, f32);
    chol_series_step(am, xs, xs32, ps, K, false, f32);
    if (tid < K) {
      const double r = 1.0 + xs[tid + kS1Ld * tid];
      xs[tid + kS1Ld * tid] = r;
      rd2[tid] = rcp_f64(r);
    }
    __syncthreads();
    rows_solve(ys, nr, K, xs, rd2, rd2);
  } else {
    if (!cta_ldl(am, K, dinv, false)) {
      if (blockIdx.x == 0 && tid == 0) *a.flag = 1;
      return;
    }
    if (tid < K) {
      rd2[tid] = rsqrt_f64(am[tid + kS1Ld * tid]);
      rdq[tid] = rd2[tid] * rd2[tid];
    }
    __syncthreads();
    for (int e = tid; e < K * K; e += nthr) {  // R2 explicitly, for R = R2 R1
      const int i = e % K, l = e / K;
      xs[i + kS1Ld * l] = i <= l ? am[i + kS1Ld * l] * rd2[i] : 0.0;
    }
    rows_solve(ys, nr, K, am, rdq, rd2);
  }
  __syncthreads();
  // Q~: column-major, or back into the core's layout (each CTA writes only the rows it read)
  for (int x = tid; x < nr * K; x += nthr) {
    const int rr = x % nr, c = x / nr, row = r0 + rr;
    if (a.core_out)
      a.core0[ycore(row, c, I1, K)] = ys[rr * ld + c];
    else
      a.Qout[row + (size_t)m * c] = ys[rr * ld + c];
  }
  // R~ = R2 R1 (both upper): column l by CTA l (every CTA holds both factors)
  if (tid < 32)
    for (int l = blockIdx.x; l < K; l += gridDim.x) {
      const int i = tid;
      if (i >= K) continue;
      double s0 = 0.0;
      for (int q = i; q <= l; ++q) s0 = fma(xs[i + kS1Ld * q], r1s[q + kS1Ld * l], s0);
      a.Rout[i + K * l] = s0;
    }
}

}  // namespace

// CholeskyQR2 of the site-1 matrix of core0 (1, I1, K, t) in one cooperative launch: Q~ to Qout
// (column-major (I1 t) x K) or, with core_out, back into core0 (1, I1, K, t); R~ (K x K) to Rout;
// *flag (device) = 1 when the caller must fall back to Householder (core0 is then unchanged).
// t_dev: when not null the rank is read there on the device and t is only its upper bound.
// gate: when not null, the kernel does nothing unless *gate != 0 on the device.
// Scratch: Q1 (q1cap doubles, at least (I1 t) K), G (K x K). *launched = false (nothing queued)
// when the sizes are outside the kernel's layout (K > 32, more rows than the grid holds) or the
// scratch is too small.
int site1_cholqr2(cudaStream_t s, double *core0, int64_t I1, int64_t K, int64_t t, const int64_t *t_dev, bool core_out,
                  const int *gate, double *Q1, int64_t q1cap, double *G, double *Rout, double *Qout, int *flag,
                  unsigned *bar, bool *launched) {
  *launched = false;
  const int64_t m = I1 * t;
  if (K < 1 || K > kS1MaxK || m < K || m * K > q1cap) return TNR_OK;
  int dev = 0, sms = 0;
  TNR_CK(cudaGetDevice(&dev));
  TNR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t nblk = std::min<int64_t>(64, sms);
  const int64_t rpc = cdiv(m, nblk);  // the device's rows per CTA never exceed this
  if (rpc > kS1MaxRowsPerCta) return TNR_OK;
  const size_t smem = sizeof(double) * (size_t)(rpc * (K + 1) + 2 * kS1Tile * kS1Chunk);
  TNR_TRY(ensure_dynamic_smem((const void *)k_site1_cholqr2, smem));
  Site1Args a;
  a.core0 = core0;
  a.t_dev = t_dev;
  a.I1 = (int)I1;
  a.K = (int)K;
  a.t = (int)t;
  a.core_out = core_out ? 1 : 0;
  a.gate = gate;
  a.Q1 = Q1;
  a.G = G;
  a.Rout = Rout;
  a.Qout = Qout;
  a.flag = flag;
  a.bar = bar;
  a.status = status_ptr();
  TNR_CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  {
    LaunchScope ls(K_QR, s);
    void *args[] = {&a};
    TNR_CK(cudaLaunchCooperativeKernel((const void *)k_site1_cholqr2, dim3((unsigned)nblk), dim3(kS1Threads), args,
                                       smem, s));
  }
  stats_work(K_QR, 2.0 * (2.0 * (double)m * K * (K + 1) / 2.0 + (double)m * K * K) + (double)K * K * K / 3.0);
  *launched = true;
  return TNR_OK;
}

}  // namespace tnr
