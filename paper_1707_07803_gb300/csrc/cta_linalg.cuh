// One-CTA dense FP64 building blocks (Householder QR, reflector application, small GEMMs, a
// symmetric Gram product and a lambda_min bound) for kernels in which one CTA of kStepThreads
// threads works through a whole factorisation: the fused rounding sweeps and the persistent
// batched solver. Operands may sit in shared or global memory.
#pragma once

#include "svd_step.cuh"

namespace tnr {

// GB300 issues FP64 at 1/64 of the FP32 rate: one FP64 warp instruction holds a sub-partition's
// FP64 pipe for ~70 cycles whether 1 or 32 lanes are active. The helpers below therefore keep the
// FP64 instruction count per CTA close to the arithmetic itself: partial sums are reduced only by
// warps that own rows, scalar work (final sums, reflector parameters) is done once by one thread
// or lane-parallel in one warp, and results are broadcast through shared memory.

// Number of warps owning at least one of `rows` rows when row r goes to thread r % kStepThreads.
static __device__ __forceinline__ int active_warps(int rows) {
  const int w = (rows + 31) >> 5;
  return w < kStepWarps ? w : kStepWarps;
}

// Sum over the CTA of per-thread values of the first `rows` threads' strided rows; the total is
// returned to every thread. red: kStepWarps doubles.
static __device__ __forceinline__ double cta_sum(double v, int rows, double *red, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = active_warps(rows);
  if (warp < nw) {
    v = dwarp_sum(v);
    if (lane == 0) red[warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    *out = t;
  }
  __syncthreads();
  return *out;
}

// Apply H = I - tau v v^T (v_i = 1 implicit, v_r stored for r > i) to rows i..m-1 of columns
// j0..j1-1 of A (ld lda). diag_zero: A(i, j) is known to be 0 (explicit-Q formation). Columns go
// in chunks of 8: each thread accumulates its rows' partial dot products for the chunk, active
// warps reduce them by shuffles, and lanes 0..7 of warp 0 finish one column each.
// red: 8 * kStepWarps doubles; wsh: 8 doubles.
static __device__ void cta_reflect(const double *v, int i, int m, double tau, double *A, int lda, int j0, int j1,
                            bool diag_zero, double *red, double *wsh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int below = m - i - 1;
  const int nw = active_warps(below);
  for (int jc = j0; jc < j1; jc += 8) {
    const int nc = j1 - jc < 8 ? j1 - jc : 8;
    if (warp < nw) {
      double p[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) p[c] = 0.0;
      for (int r = i + 1 + threadIdx.x; r < m; r += kStepThreads) {
        const double vr = v[r];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c < nc) p[c] = fma(vr, A[r + lda * (jc + c)], p[c]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c < nc) {
          const double s = dwarp_sum(p[c]);
          if (lane == 0) red[warp * 8 + c] = s;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < nc) {
      const int c = threadIdx.x;
      double *aij = A + i + lda * (jc + c);
      double w = diag_zero ? 0.0 : *aij;
      for (int q = 0; q < nw; ++q) w += red[q * 8 + c];
      w *= tau;
      wsh[c] = w;
      *aij = diag_zero ? -w : *aij - w;
    }
    __syncthreads();
    if (warp < nw) {
      double wc[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) wc[c] = c < nc ? wsh[c] : 0.0;
      for (int r = i + 1 + threadIdx.x; r < m; r += kStepThreads) {
        const double vr = v[r];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c < nc) A[r + lda * (jc + c)] = fma(-wc[c], vr, A[r + lda * (jc + c)]);
      }
    }
    // the next chunk writes red and wsh only after its own first barrier
  }
  __syncthreads();
}

// Householder QR of A (m x n, ld m, shared memory): A <- Q (m x nq explicit, nq = min(m, n)),
// R (nq x n, ld nq, upper trapezoidal) -> Rout. tau: nq doubles; red: 8 * kStepWarps doubles;
// sc: 8 doubles of broadcast scratch.
static __device__ void cta_qr(double *A, int m, int n, double *Rout, double *tau, double *red, double *sc) {
  const int nq = m < n ? m : n;
  for (int i = 0; i < nq; ++i) {
    double *col = A + m * i;
    double s = 0.0;
    for (int r = i + 1 + threadIdx.x; r < m; r += kStepThreads) s = fma(col[r], col[r], s);
    const double sig = cta_sum(s, m - i - 1, red, sc);
    if (threadIdx.x == 0) {  // reflector parameters once, broadcast through shared memory
      const double alpha = col[i];
      double tv = 0.0, beta = alpha, scal = 0.0;
      if (sig > 0.0) householder_params(alpha, sig, beta, tv, scal);
      col[i] = beta;
      tau[i] = tv;
      sc[1] = scal;
    }
    __syncthreads();
    const double tv = tau[i];
    if (tv != 0.0) {
      const double scal = sc[1];
      for (int r = i + 1 + threadIdx.x; r < m; r += kStepThreads) col[r] *= scal;
      __syncthreads();
      cta_reflect(col, i, m, tv, A, m, i + 1, n, false, red, sc);
    }
  }
  for (int idx = threadIdx.x; idx < nq * n; idx += kStepThreads) {
    const int r = idx % nq, c = idx / nq;
    Rout[idx] = r <= c ? A[r + m * c] : 0.0;
  }
  __syncthreads();
  // explicit Q (backward accumulation): H_i applied to columns i+1..nq-1, whose row i is 0
  for (int i = nq - 1; i >= 0; --i) {
    const double tv = tau[i];
    double *col = A + m * i;
    if (tv != 0.0) cta_reflect(col, i, m, tv, A, m, i + 1, nq, true, red, sc);
    for (int q = threadIdx.x; q < m; q += kStepThreads) col[q] = q < i ? 0.0 : (q == i ? 1.0 - tv : -tv * col[q]);
    __syncthreads();
  }
}

// C (m x n, ld m) = A (m x k, ld lda) B (k x n, ld ldb); C aliases neither.
static __device__ void cta_gemm(double *C, const double *A, int lda, const double *B, int ldb, int m, int n, int k) {
  for (int idx = threadIdx.x; idx < m * n; idx += kStepThreads) {
    const int i = idx % m, j = idx / m;
    const double *a = A + i;
    const double *b = B + ldb * j;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int l = 0;
    for (; l + 3 < k; l += 4) {
      s0 = fma(a[lda * l], b[l], s0);
      s1 = fma(a[lda * (l + 1)], b[l + 1], s1);
      s2 = fma(a[lda * (l + 2)], b[l + 2], s2);
      s3 = fma(a[lda * (l + 3)], b[l + 3], s3);
    }
    for (; l < k; ++l) s0 = fma(a[lda * l], b[l], s0);
    C[idx] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
}

// C (rows x t, ld rows) <- C US (US: t x r, ld t, r <= t) in place, in blocks of rows staged in
// tmp (cap doubles): output row i depends only on input row i, and keeps leading dimension rows.
static __device__ void cta_absorb_right(double *C, int rows, int t, const double *US, int r, double *tmp, int cap) {
  int rb = cap / t;
  if (rb > rows) rb = rows;
  for (int r0 = 0; r0 < rows; r0 += rb) {
    const int nb = rows - r0 < rb ? rows - r0 : rb;
    for (int idx = threadIdx.x; idx < nb * t; idx += kStepThreads) {
      const int i = idx % nb, l = idx / nb;
      tmp[idx] = C[r0 + i + rows * l];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * r; idx += kStepThreads) {
      const int i = idx % nb, c = idx / nb;
      const double *u = US + t * c;
      double s0 = 0.0, s1 = 0.0;
      int l = 0;
      for (; l + 1 < t; l += 2) {
        s0 = fma(tmp[i + nb * l], u[l], s0);
        s1 = fma(tmp[i + nb * (l + 1)], u[l + 1], s1);
      }
      if (l < t) s0 = fma(tmp[i + nb * l], u[l], s0);
      C[r0 + i + rows * c] = s0 + s1;
    }
    __syncthreads();
  }
}

// G (r x r, symmetric) = A^T B for A, B (m x r, ld m) with A^T B known to be symmetric: one warp
// per entry i <= j (lanes stride the reduction), mirrored.
static __device__ void cta_tn_sym(double *G, const double *A, const double *B, int m, int r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int E = r * (r + 1) / 2;
  for (int e = warp; e < E; e += kStepWarps) {
    int j = 0, base = 0;
    while (base + j + 1 <= e) {
      base += j + 1;
      ++j;
    }
    const int i = e - base;
    const double *ai = A + m * i, *bj = B + m * j;
    double s0 = 0.0, s1 = 0.0;
    int l = lane;
    for (; l + 32 < m; l += 64) {
      s0 = fma(ai[l], bj[l], s0);
      s1 = fma(ai[l + 32], bj[l + 32], s1);
    }
    if (l < m) s0 = fma(ai[l], bj[l], s0);
    const double v = dwarp_sum(s0 + s1);
    if (lane == 0) {
      G[i + r * j] = v;
      G[j + r * i] = v;
    }
  }
  __syncthreads();
}

// Lower bound on lambda_min of a symmetric r x r matrix G (r <= 32, in place), one warp:
// G = L D L^T (unit lower L, no pivoting) and lambda_min >= 1 / trace(G^{-1}), trace(G^{-1}) =
// sum_i d_i^{-1} sum_c (L^{-1})_{ic}^2. Returns 0 when a pivot is not positive and finite
// (no bound). Lanes own rows during the factorisation and columns of L^{-1} afterwards.
static __device__ double warp_lambda_min_bound(double *G, int r) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int j = 0; j < r; ++j) {
    const double dj = G[j + r * j];
    if (!(dj > 0.0) || !isfinite(dj)) {
      ok = false;
      break;
    }
    const double inv = rcp_f64(dj);  // Newton-refined reciprocal (no FP64 division sequence)
    double gij = 0.0;
    if (lane > j && lane < r) {
      gij = G[lane + r * j];
      for (int l = j + 1; l <= lane; ++l) G[lane + r * l] = fma(-gij * inv, G[l + r * j], G[lane + r * l]);
    }
    __syncwarp();
    if (lane > j && lane < r) G[lane + r * j] = gij * inv;  // L(i, j)
    if (lane == j) G[j + r * j] = inv;                      // 1 / d_j on the diagonal
    __syncwarp();
  }
  if (!__all_sync(0xffffffffu, ok)) return 0.0;
  // column `lane` of L^{-1}: x_c = 1, x_i = -sum_{l=c}^{i-1} L(i, l) x_l; sum of x_i^2 / d_i
  double tr = 0.0;
  if (lane < r) {
    double x[32];
    x[lane] = 1.0;
    tr = G[lane + r * lane];
    for (int i = lane + 1; i < r; ++i) {
      double acc = 0.0;
      for (int l = lane; l < i; ++l) acc = fma(-G[i + r * l], x[l], acc);
      x[i] = acc;
      tr = fma(acc * acc, G[i + r * i], tr);
    }
  }
  tr = dwarp_sum(tr);
  return (tr > 0.0 && isfinite(tr)) ? 1.0 / tr : 0.0;
}

}  // namespace tnr
