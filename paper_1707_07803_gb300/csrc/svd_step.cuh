// Truncated-SVD step of the right-to-left rounding sweep (Alg. 5.2 loop with the rounding of
// Section 5.4) as a device function run by one whole CTA of kStepThreads threads, with every
// operand in shared or global memory. Used by the one-step kernel (sweep_small.cu) and by the
// fused rounding kernel (round_small.cu).
//
// For the core M (t x w, column-major, ld t) of site k:
//   X = M (t >= w) or M^T (t < w), n = min(t, w); Householder QR X = Q_x R;
//   one-sided Jacobi SVD of G = R (t >= w) or R^T (t < w): G V = U S;
//   the kept rank r (truncation rule of the rounding: smallest r >= 1 with
//   sum_{l >= r} s_l^2 <= delta2 = tol^2 ||Y||^2 / (d - 1), then r <= max_rank);
//   the new core V_M[:, :r]^T (r x w, orthonormal rows) and U_M[:, :r] diag(S) (t x r, ld t),
//   where (t >= w): U_M = Q_x U, V_M = V;  (t < w): U_M = U, V_M = Q_x V.
// Q_x stays implicit (its reflectors are applied to the r kept columns only). core_out may alias
// M; US aliases neither. work holds svd_step_work(t, w) doubles. Returns r (all threads).
#pragma once

#include <cfloat>
#include <cmath>

#include "dev_common.cuh"
#include "jacobi.cuh"
#include "tnr_internal.cuh"

namespace tnr {

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;
constexpr int kStepMaxN = 1024;  // largest min(t, w)

static __host__ __device__ inline int64_t svd_step_work(int64_t t, int64_t w) {
  const int64_t mm = t >= w ? t : w, n = t >= w ? w : t, jw = jacobi_mixed_work(n);
  return mm * n + 2 * n * n + 2 * n + (mm * n > jw ? mm * n : jw);
}

static __device__ __noinline__ int svd_step_cta(const double *M, int t, int w, double delta2, int64_t max_rank,
                                         double *core_out, double *US, double *work, int *status) {
  const bool tall = t >= w;
  const int mm = tall ? t : w, n = tall ? w : t;
  double *X = work;          // mm x n (ld mm): Householder vectors below the diagonal, R above
  double *G = X + mm * n;    // n x n
  double *V = G + n * n;     // n x n
  double *tau = V + n * n;   // n
  double *nrm = tau + n;     // n (Jacobi column norms, then singular values)
  double *W = nrm + n;       // mm x n: reflector application workspace, then the work area of
                             // the mixed-precision Jacobi (jacobi_mixed_work(n) doubles)
  __shared__ int s_r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < mm * n; idx += kStepThreads) {
    const int i = idx % mm, j = idx / mm;
    X[idx] = tall ? M[i + t * j] : M[j + t * i];
  }
  __syncthreads();
  // ---- Householder QR of X (mm x n), reflectors left in X
  for (int i = 0; i < n; ++i) {
    if (warp == 0) {
      double *col = X + mm * i;
      double sig = 0.0, sig1 = 0.0;
      int r0 = i + 1 + lane;
      for (; r0 + 32 < mm; r0 += 64) {  // two rows in flight per lane
        sig = fma(col[r0], col[r0], sig);
        sig1 = fma(col[r0 + 32], col[r0 + 32], sig1);
      }
      if (r0 < mm) sig = fma(col[r0], col[r0], sig);
      sig = dwarp_sum(sig + sig1);
      const double alpha = col[i];
      double tv = 0.0, beta = alpha, scal = 0.0;
      if (sig > 0.0) {
        householder_params(alpha, sig, beta, tv, scal);
      }
      for (int r = i + 1 + lane; r < mm; r += 32) col[r] *= scal;
      __syncwarp();
      if (lane == 0) {
        col[i] = beta;
        tau[i] = tv;
      }
    }
    __syncthreads();
    const double tv = tau[i];
    const double *v = X + mm * i;
    if (tv != 0.0) {
      for (int j = i + 1 + warp; j < n; j += kStepWarps) {
        double *col = X + mm * j;
        double s = lane == 0 ? col[i] : 0.0, s1 = 0.0;
        int r = i + 1 + lane;
        for (; r + 32 < mm; r += 64) {  // two rows in flight per lane
          s = fma(v[r], col[r], s);
          s1 = fma(v[r + 32], col[r + 32], s1);
        }
        if (r < mm) s = fma(v[r], col[r], s);
        s = dwarp_sum(s + s1) * tv;
        if (lane == 0) col[i] -= s;
        r = i + 1 + lane;
        for (; r + 32 < mm; r += 64) {  // loads of both rows before the stores
          const double c0 = col[r], c1 = col[r + 32], v0 = v[r], v1 = v[r + 32];
          col[r] = fma(-s, v0, c0);
          col[r + 32] = fma(-s, v1, c1);
        }
        if (r < mm) col[r] = fma(-s, v[r], col[r]);
      }
    }
    __syncthreads();
  }
  // ---- G = R (tall) or R^T, V = I
  for (int idx = threadIdx.x; idx < n * n; idx += kStepThreads) {
    const int i = idx % n, j = idx / n;
    const double rij = i <= j ? X[i + mm * j] : 0.0;        // R(i, j)
    const double rji = j <= i ? X[j + mm * i] : 0.0;        // R(j, i)
    G[idx] = tall ? rij : rji;
    V[idx] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  // ---- no-truncation certificate. The SVD here only decides truncation (Alg. 5.2's own step is
  // the RQ factorisation M = L Q). sigma_min(M) = sigma_min(R) >= 1 / ||R^{-1}||_F; when that bound
  // already exceeds delta and the rank cap does not bind, no singular value can be discarded and
  // the factors of the QR are returned directly (same rounded tensor, no Jacobi iterations):
  //   tall: core = I_w (r = w), U S = M;   wide: core = Q_x^T (r = t), U S = R^T.
  __shared__ int s_nocut;
  if (warp == 0) {
    int ok = 0;
    if (n <= 32 && (max_rank <= 0 || n <= max_rank)) {
      // column `lane` of R^{-1} by back substitution (R upper triangular, X holds R), with the
      // reciprocals of the diagonal formed once, lane-parallel (one FP64 division sequence)
      __shared__ double s_dinv[32];
      bool bad = false;
      if (lane < n) {
        const double dg = X[lane + mm * lane];
        bad = dg == 0.0 || !isfinite(dg);
        s_dinv[lane] = bad ? 0.0 : 1.0 / dg;
      }
      __syncwarp();
      const bool anybad = __any_sync(0xffffffffu, bad);
      double colsq = 0.0;
      if (!anybad && lane < n) {
        double x[32];
        for (int i = lane; i >= 0; --i) {
          double acc = (i == lane) ? 1.0 : 0.0;
          for (int l = i + 1; l <= lane; ++l) acc = fma(-X[i + mm * l], x[l], acc);
          x[i] = acc * s_dinv[i];
          colsq = fma(x[i], x[i], colsq);
        }
      }
      const double inv2 = dwarp_sum(colsq);  // ||R^{-1}||_F^2
      // sigma_min^2 >= 1 / inv2 > delta2 (with a relative margin for the rounding of inv2)
      ok = (!anybad && isfinite(inv2) && inv2 > 0.0 && inv2 * delta2 * (1.0 + 1e-6) < 1.0) ? 1 : 0;
    }
    if (lane == 0) s_nocut = ok;
  }
  __syncthreads();
  if (s_nocut) {
    if (tall) {  // r = w: core = I_w, U S = M (M itself is unchanged by the QR)
      for (int idx = threadIdx.x; idx < t * w; idx += kStepThreads) US[idx] = M[idx];
      __syncthreads();
      for (int idx = threadIdx.x; idx < w * w; idx += kStepThreads) core_out[idx] = (idx % w == idx / w) ? 1.0 : 0.0;
      __syncthreads();
      return w;
    } else {  // r = t: core = Q_x^T (t x w), U S = R^T (t x t)
      for (int idx = threadIdx.x; idx < mm * n; idx += kStepThreads) {
        const int i = idx % mm, c = idx / mm;
        W[idx] = (i == c) ? 1.0 : 0.0;
      }
      __syncthreads();
      for (int i = n - 1; i >= 0; --i) {  // W <- H_i W
        const double tv = tau[i];
        if (tv != 0.0) {
          const double *v = X + mm * i;
          for (int c = warp; c < n; c += kStepWarps) {
            double *col = W + mm * c;
            double s = lane == 0 ? col[i] : 0.0;
            for (int q = i + 1 + lane; q < mm; q += 32) s = fma(v[q], col[q], s);
            s = dwarp_sum(s) * tv;
            if (lane == 0) col[i] -= s;
            for (int q = i + 1 + lane; q < mm; q += 32) col[q] = fma(-s, v[q], col[q]);
          }
        }
        __syncthreads();
      }
      for (int idx = threadIdx.x; idx < t * t; idx += kStepThreads) {
        const int i = idx % t, c = idx / t;
        US[idx] = i >= c ? X[c + mm * i] : 0.0;  // R^T(i, c) = R(c, i)
      }
      for (int idx = threadIdx.x; idx < t * w; idx += kStepThreads) {
        const int c = idx % t, j = idx / t;
        core_out[idx] = W[j + mm * c];
      }
      __syncthreads();
      return t;
    }
  }
  // ---- one-sided Jacobi on G (jacobi.cuh): FP32-preconditioned, finished in FP64
  jacobi_sweeps_mixed(G, V, n, nrm, W);
  // ---- singular values (column norms of G, one thread per column), order, truncation
  for (int j = threadIdx.x; j < n; j += kStepThreads) {
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < n; i += 2) {
      s0 = fma(G[i + n * j], G[i + n * j], s0);
      s1 = fma(G[i + 1 + n * j], G[i + 1 + n * j], s1);
    }
    if (i < n) s0 = fma(G[i + n * j], G[i + n * j], s0);
    nrm[j] = sqrt(s0 + s1);
  }
  __syncthreads();
  // s_order[rank] = column of G holding the rank-th largest singular value (stable)
  __shared__ int s_order[kStepMaxN];
  for (int j = threadIdx.x; j < n; j += kStepThreads) {
    const double sj = nrm[j];
    int rk = 0;
    for (int i = 0; i < n; ++i) {
      const double si = nrm[i];
      rk += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    s_order[rk] = (int)j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tail = 0.0;
    int r = n;
    for (int cand = n - 1; cand >= 1; --cand) {
      const double sv = nrm[s_order[cand]];
      tail += sv * sv;
      if (tail <= delta2)
        r = cand;
      else
        break;
    }
    bool bad = false;
    for (int l = 0; l < n; ++l) bad |= !isfinite(nrm[l]);
    if (bad) set_status(status, TNR_ENONFINITE);
    if (max_rank > 0 && r > max_rank) r = (int)max_rank;
    if (r < 1) r = 1;
    s_r = (int)r;
  }
  __syncthreads();
  const int r = s_r;
  // ---- outputs
  // left factor U_G[:, :r] diag(S) = G[:, order[:r]] (the Jacobi columns are U_G S), right
  // factor V[:, order[:r]]. One of them is mapped through Q_x: W (mm x r) = Q_x [Z; 0].
  // tall : Z = G[:, order[:r]] -> US = Q_x Z (t x r); core = V[:, order]^T (r x w)
  // wide : Z = V[:, order[:r]] -> core = (Q_x Z)^T (r x w); US = G[:, order] (t x r)
  for (int idx = threadIdx.x; idx < mm * r; idx += kStepThreads) {
    const int i = idx % mm, c = idx / mm;
    const int col = s_order[c];
    W[idx] = i < n ? (tall ? G[i + n * col] : V[i + n * col]) : 0.0;
  }
  __syncthreads();
  for (int i = n - 1; i >= 0; --i) {  // W <- H_i W, i = n-1 .. 0
    const double tv = tau[i];
    if (tv == 0.0) continue;
    const double *v = X + mm * i;
    for (int c = warp; c < r; c += kStepWarps) {
      double *col = W + mm * c;
      double s = lane == 0 ? col[i] : 0.0, s1 = 0.0;
      int q = i + 1 + lane;
      for (; q + 32 < mm; q += 64) {  // two rows in flight per lane
        s = fma(v[q], col[q], s);
        s1 = fma(v[q + 32], col[q + 32], s1);
      }
      if (q < mm) s = fma(v[q], col[q], s);
      s = dwarp_sum(s + s1) * tv;
      if (lane == 0) col[i] -= s;
      q = i + 1 + lane;
      for (; q + 32 < mm; q += 64) {  // loads of both rows before the stores
        const double c0 = col[q], c1 = col[q + 32], v0 = v[q], v1 = v[q + 32];
        col[q] = fma(-s, v0, c0);
        col[q + 32] = fma(-s, v1, c1);
      }
      if (q < mm) col[q] = fma(-s, v[q], col[q]);
    }
    __syncthreads();
  }
  if (tall) {
    for (int idx = threadIdx.x; idx < t * r; idx += kStepThreads) US[idx] = W[idx];  // t x r, ld t = mm
    for (int idx = threadIdx.x; idx < r * w; idx += kStepThreads) {
      const int c = idx % r, j = idx / r;
      core_out[idx] = V[j + n * s_order[c]];
    }
  } else {
    for (int idx = threadIdx.x; idx < r * w; idx += kStepThreads) {
      const int c = idx % r, j = idx / r;
      core_out[idx] = W[j + mm * c];
    }
    for (int idx = threadIdx.x; idx < t * r; idx += kStepThreads) {
      const int i = idx % t, c = idx / t;
      US[idx] = G[i + n * s_order[c]];
    }
  }
  __syncthreads();
  return r;
}

}  // namespace tnr
