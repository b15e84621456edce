// Symmetric Gram kernel for tall row-major matrices (element (r, c) at c + K r), the first step of
// the sparse solver's CholeskyQR (the site-1 CholeskyQR2 of the MPO solver is site1_qr.cu).
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

}  // namespace
}  // namespace tnr
