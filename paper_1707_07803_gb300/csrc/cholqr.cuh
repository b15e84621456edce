// CholeskyQR pieces for tall row-major matrices (element (r, c) at c + K r), shared by the sparse
// solver and the site-1 step of the MPO solver: a symmetric Gram kernel, a one-CTA Cholesky for
// K <= 32 with one thread per matrix element, and a warp-per-row triangular solve. Cholesky
// QR trades the Householder reflector chain (one dependent step per column, each a chain of FP64
// instructions on GB300's 1/64-rate FP64 pipe) for a Gram matrix, K pivots and a solve.
#pragma once

#include <algorithm>

#include "dev_common.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

// G (K x K, column-major, zeroed by the caller) += Y^T Y for Y row-major (n x K): chunks of rows are
// staged in shared memory and each thread accumulates a few (i <= j) pairs, exploiting symmetry
// (half the FP64 work of a GEMM); the partial sums are added into G with atomics and mirrored.
constexpr int kGramRows = 64;
constexpr int kGramThreads = 512;
constexpr int kGramPairs = 5;  // pairs per thread: K (K + 1) / 2 <= 5 * 512 (K <= 70)

__global__ void __launch_bounds__(kGramThreads) k_gram_rm(const double *__restrict__ Y, int64_t n, int64_t K, double *G) {
  extern __shared__ double ys[];  // kGramRows x K
  const int64_t npairs = K * (K + 1) / 2;
  int pi[kGramPairs], pj[kGramPairs];
  double acc[kGramPairs];
#pragma unroll
  for (int u = 0; u < kGramPairs; ++u) {
    const int64_t pr = threadIdx.x + (int64_t)u * kGramThreads;
    int j = 0, base = 0;
    if (pr < npairs)
      while (base + j + 1 <= pr) {
        base += j + 1;
        ++j;
      }
    pi[u] = pr < npairs ? (int)(pr - base) : -1;
    pj[u] = j;
    acc[u] = 0.0;
  }
  for (int64_t r0 = (int64_t)blockIdx.x * kGramRows; r0 < n; r0 += (int64_t)gridDim.x * kGramRows) {
    const int64_t nr = n - r0 < kGramRows ? n - r0 : kGramRows;
    for (int64_t x = threadIdx.x; x < nr * K; x += kGramThreads) ys[x] = Y[r0 * K + x];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kGramPairs; ++u) {
      if (pi[u] < 0) continue;
      const double *a = ys + pi[u], *b = ys + pj[u];
      double s0 = acc[u];
      for (int64_t rr = 0; rr < nr; ++rr) s0 = fma(a[rr * K], b[rr * K], s0);
      acc[u] = s0;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kGramPairs; ++u) {
    if (pi[u] < 0) continue;
    atomicAdd(&G[pi[u] + K * pj[u]], acc[u]);
    if (pi[u] != pj[u]) atomicAdd(&G[pj[u] + K * pi[u]], acc[u]);
  }
}

// Cholesky G = R^T R of a K x K matrix (K <= 32, column-major) in one CTA of 1024 threads, one
// thread per element, in the square-root-free form G = U^T D U (U unit upper): per pivot one
// reciprocal of d_j (FP32 seed + Newton, on one thread) and one fused trailing update
// a_il -= a_ji a_jl / d_j; R = D^{1/2} U at the end, all rows at once. Writes R (upper, zeros
// below) and rdiag = 1 / diag(R); on a pivot that is not positive and finite it sets *flag = 1.
// near_identity (second CholeskyQR pass): G must be within 0.5 / K of the identity entrywise,
// i.e. the first pass left a well-conditioned factor (||G - I||_2 < 1/2); otherwise *flag = 1.
// This is the regime (cond(Y) below ~1e8) in which CholeskyQR2 is orthogonal to rounding level.
__global__ void __launch_bounds__(1024) k_chol_small(const double *__restrict__ G, int K, double *Rout, double *rdiag,
                                                     int *flag, int near_identity) {
  __shared__ double a[32 * 32];
  __shared__ double s_dinv[32];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  const bool own = tid < K * K;
  const int i = tid % K, l = tid / K;  // warp l holds column l
  if (own) a[tid] = G[tid];
  if (tid == 0) s_bad = 0;
  __syncthreads();
  if (near_identity && own) {
    const double dev = fabs(a[tid] - (i == l ? 1.0 : 0.0));
    if (!(dev <= 0.5 / K)) s_bad = 1;  // benign race: every writer stores 1
  }
  __syncthreads();
  for (int j = 0; j < K && !s_bad; ++j) {
    if (tid == 0) {
      const double dj = a[j + K * j];
      if (!(dj > 0.0) || !isfinite(dj))
        s_bad = 1;
      else
        s_dinv[j] = rcp_f64(dj);
    }
    __syncthreads();
    if (s_bad) break;
    // a_il -= a_ji a_jl / d_j for j < i <= l (upper triangle; row j stays unscaled)
    if (own && l > j && i > j && i <= l) a[tid] = fma(-a[j + K * i] * s_dinv[j], a[j + K * l], a[tid]);
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) *flag = 1;
    return;
  }
  // R(j, l) = a_jl / sqrt(d_j): rdiag[j] = 1 / sqrt(d_j)
  if (tid < K) rdiag[tid] = rsqrt_f64(a[tid + K * tid]);
  __syncthreads();
  if (own) {
    const double rj = rsqrt_f64(a[i + K * i]);
    Rout[tid] = i <= l ? a[tid] * rj : 0.0;
  }
}

// Y (n x K, row-major, K <= 32) <- Y R^{-1} for R upper: one warp per row, lane c owns column c;
// step j: lane j finishes x_j = y_j / R_jj, broadcasts it, lanes c > j subtract x_j R_jc.
__global__ void k_trsm_warp(double *Y, int64_t n, int K, const double *__restrict__ R, const double *__restrict__ rdiag) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double rl[32];  // column `lane` of R: rl[j] = R(j, lane)
#pragma unroll
  for (int j = 0; j < 32; ++j) rl[j] = (lane < K && j < K) ? R[j + K * lane] : 0.0;
  const double rd = lane < K ? rdiag[lane] : 0.0;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    double y = lane < K ? Y[r * K + lane] : 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= K) break;
      const double xj = __shfl_sync(0xffffffffu, y * rd, j);
      if (lane == j) y = xj;
      else if (lane > j) y = fma(-xj, rl[j], y);
    }
    if (lane < K) Y[r * K + lane] = y;
  }
}

// One CholeskyQR pass on row-major Y (n x K, K <= 32): G = Y^T Y, G = R^T R, Y <- Y R^{-1}.
// second: the pass of CholeskyQR2 that checks that G is near the identity.
int cholqr_pass_small(cudaStream_t s, double *Y, int64_t n, int K, double *G, double *R, double *rdiag, int *flag,
                      int kclass, bool second) {
  TNR_CK(cudaMemsetAsync(G, 0, sizeof(double) * K * K, s));
  const size_t smem = sizeof(double) * kGramRows * K;
  TNR_TRY(ensure_dynamic_smem((const void *)k_gram_rm, smem));
  LaunchScope ls(kclass, s);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(cdiv(n, kGramRows), 152 * 4));
  k_gram_rm<<<(unsigned)blocks, kGramThreads, smem, s>>>(Y, n, K, G);
  k_chol_small<<<1, 1024, 0, s>>>(G, K, R, rdiag, flag, second ? 1 : 0);
  const int64_t tblocks = std::max<int64_t>(1, std::min<int64_t>(cdiv(n * 32, 256), 152 * 16));
  k_trsm_warp<<<(unsigned)tblocks, 256, 0, s>>>(Y, n, K, R, rdiag);
  stats_work(kclass, 2.0 * (double)n * K * K + (double)K * K * K / 3.0);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

}  // namespace
}  // namespace tnr
