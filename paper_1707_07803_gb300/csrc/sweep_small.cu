// Fused truncated-SVD step of the right-to-left rounding sweep (Alg. 5.2 loop with the
// rounding of Section 5.4), for cores that fit one CTA's shared memory.
//
// For the core M (t x w, column-major) of site k it computes, in one launch:
//   X = M (t >= w) or M^T (t < w), n = min(t, w); Householder QR X = Q_x R;
//   one-sided Jacobi SVD of G = R (t >= w) or R^T (t < w): G V = U S;
//   the kept rank r (truncation rule of the rounding: smallest r >= 1 with
//   sum_{l >= r} s_l^2 <= tol^2 ||Y||^2 / (d - 1), then r <= max_rank);
//   the new core V_M[:, :r]^T (r x w, orthonormal rows) and U_M[:, :r] diag(S) (t x r), where
//   (t >= w): U_M = Q_x U, V_M = V;  (t < w): U_M = U, V_M = Q_x V.
// Q_x stays implicit (its reflectors are applied to the r kept columns only).
#include <cfloat>
#include <cmath>

#include "dev_common.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

constexpr int kSvdThreads = 256;
constexpr int kSvdWarps = kSvdThreads / 32;

struct SvdStepArgs {
  const double *M;  // t x w, ld t
  int64_t t, w;
  const double *norm2;  // ||Y||_F^2 (device)
  double tol;
  int64_t dm1, max_rank;
  double *core_out;  // r x w, ld r (may alias M)
  double *US;        // t x r, ld t
  int64_t *r_out;
  int *status;
};

__global__ void __launch_bounds__(kSvdThreads) k_svd_step(SvdStepArgs a) {
  extern __shared__ double sm[];
  const int t = (int)a.t, w = (int)a.w;
  const bool tall = t >= w;
  const int mm = tall ? t : w, n = tall ? w : t;
  double *X = sm;            // mm x n (ld mm): Householder vectors below the diagonal, R above
  double *G = X + mm * n;    // n x n
  double *V = G + n * n;     // n x n
  double *tau = V + n * n;   // n
  double *nrm = tau + n;     // n (Jacobi column norms, then singular values)
  double *W = nrm + n;       // mm x n: reflector application workspace
  __shared__ int s_r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < mm * n; idx += kSvdThreads) {
    const int i = idx % mm, j = idx / mm;
    X[idx] = tall ? a.M[i + t * j] : a.M[j + t * i];
  }
  __syncthreads();
  // ---- Householder QR of X (mm x n), reflectors left in X
  for (int i = 0; i < n; ++i) {
    if (warp == 0) {
      double *col = X + mm * i;
      double sig = 0.0;
      for (int r = i + 1 + lane; r < mm; r += 32) sig = fma(col[r], col[r], sig);
      sig = dwarp_sum(sig);
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
      for (int j = i + 1 + warp; j < n; j += kSvdWarps) {
        double *col = X + mm * j;
        double s = lane == 0 ? col[i] : 0.0;
        for (int r = i + 1 + lane; r < mm; r += 32) s = fma(v[r], col[r], s);
        s = dwarp_sum(s) * tv;
        if (lane == 0) col[i] -= s;
        for (int r = i + 1 + lane; r < mm; r += 32) col[r] = fma(-s, v[r], col[r]);
      }
    }
    __syncthreads();
  }
  // ---- G = R (tall) or R^T, V = I
  for (int idx = threadIdx.x; idx < n * n; idx += kSvdThreads) {
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
    const double delta2 = a.dm1 > 0 ? a.tol * a.tol * (*a.norm2) / (double)a.dm1 : 0.0;
    if (n <= 32 && (a.max_rank <= 0 || n <= a.max_rank)) {
      // column `lane` of R^{-1} by back substitution (R upper triangular, X holds R)
      double colsq = 0.0;
      bool bad = false;
      if (lane < n) {
        double x[32];
        for (int i = lane; i >= 0; --i) {
          double acc = (i == lane) ? 1.0 : 0.0;
          for (int l = i + 1; l <= lane; ++l) acc = fma(-X[i + mm * l], x[l], acc);
          const double d = X[i + mm * i];
          if (d == 0.0 || !isfinite(d)) {
            bad = true;
            break;
          }
          x[i] = acc / d;
          colsq = fma(x[i], x[i], colsq);
        }
      }
      const bool anybad = __any_sync(0xffffffffu, bad);
      const double inv2 = dwarp_sum(colsq);  // ||R^{-1}||_F^2
      // sigma_min^2 >= 1 / inv2 > delta2 (with a relative margin for the rounding of inv2)
      ok = (!anybad && isfinite(inv2) && inv2 > 0.0 && inv2 * delta2 * (1.0 + 1e-6) < 1.0) ? 1 : 0;
    }
    if (lane == 0) s_nocut = ok;
  }
  __syncthreads();
  if (s_nocut) {
    if (tall) {  // r = w: core = I_w, U S = M (copied before the QR overwrote nothing: read a.M)
      for (int idx = threadIdx.x; idx < t * w; idx += kSvdThreads) a.US[idx] = a.M[idx];
      __syncthreads();
      for (int idx = threadIdx.x; idx < w * w; idx += kSvdThreads) a.core_out[idx] = (idx % w == idx / w) ? 1.0 : 0.0;
      if (threadIdx.x == 0) *a.r_out = (int64_t)w;
    } else {  // r = t: core = Q_x^T (t x w), U S = R^T (t x t)
      for (int idx = threadIdx.x; idx < mm * n; idx += kSvdThreads) {
        const int i = idx % mm, c = idx / mm;
        W[idx] = (i == c) ? 1.0 : 0.0;
      }
      __syncthreads();
      for (int i = n - 1; i >= 0; --i) {  // W <- H_i W
        const double tv = tau[i];
        if (tv != 0.0) {
          const double *v = X + mm * i;
          for (int c = warp; c < n; c += kSvdWarps) {
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
      for (int idx = threadIdx.x; idx < t * t; idx += kSvdThreads) {
        const int i = idx % t, c = idx / t;
        a.US[idx] = i >= c ? X[c + mm * i] : 0.0;  // R^T(i, c) = R(c, i)
      }
      for (int idx = threadIdx.x; idx < t * w; idx += kSvdThreads) {
        const int c = idx % t, j = idx / t;
        a.core_out[idx] = W[j + mm * c];
      }
      if (threadIdx.x == 0) *a.r_out = (int64_t)t;
    }
    return;
  }
  // ---- one-sided Jacobi on G. Each column pair of a round-robin round is handled by a group
  // of g = next_pow2(min(n, 32)) lanes (lanes = rows), 32 / g pairs per warp, so the pairs of
  // a round run in parallel, row updates are lane-parallel, and the dot-product reduction tree
  // has only log2(g) levels (each level is a 64-cycle dependent FP64 add on this GPU).
  {
    const int np = (n + 1) & ~1;
    int g = 1;
    while (g < n && g < 32) g <<= 1;
    const int ppw = 32 / g, gi = lane / g, li = lane % g;
    const int pstride = kSvdWarps * ppw;
    const double tolj = 16.0 * DBL_EPSILON * sqrt((double)(n > 4 ? n : 4));
    const double tol2 = tolj * tolj;
    __shared__ double s_fro2;
    __shared__ int s_rot2;
    for (int sweep = 0; sweep < 60; ++sweep) {
      for (int j = threadIdx.x; j < n; j += kSvdThreads) {
        double s0 = 0.0, s1 = 0.0;
        int i = 0;
        for (; i + 1 < n; i += 2) {
          s0 = fma(G[i + n * j], G[i + n * j], s0);
          s1 = fma(G[i + 1 + n * j], G[i + 1 + n * j], s1);
        }
        if (i < n) s0 = fma(G[i + n * j], G[i + n * j], s0);
        nrm[j] = s0 + s1;
      }
      if (threadIdx.x == 0) s_rot2 = 0;
      __syncthreads();
      if (sweep == 0) {
        if (threadIdx.x == 0) {
          double f = 0.0;
          for (int j = 0; j < n; ++j) f += nrm[j];
          s_fro2 = f;
        }
        __syncthreads();
      }
      const double floor2 = (double)n * DBL_EPSILON * (double)n * DBL_EPSILON * s_fro2;
      for (int round = 0; round < np - 1; ++round) {
        for (int pbase = warp * ppw; pbase < np / 2; pbase += pstride) {
          const int pr = pbase + gi;
          int p = -1, q = -1;
          if (pr < np / 2) {
            if (pr == 0) {
              p = round;
              q = np - 1;
            } else {
              p = (round + pr) % (np - 1);
              q = (round - pr + (np - 1)) % (np - 1);
            }
            if (p > q) {
              const int x = p;
              p = q;
              q = x;
            }
          }
          bool act = p >= 0 && q < n;
          double al = 0.0, be = 0.0;
          if (act) {
            al = nrm[p];
            be = nrm[q];
            act = al > floor2 && be > floor2;
          }
          double ga = 0.0;
          if (act)
            for (int i = li; i < n; i += g) ga = fma(G[i + n * p], G[i + n * q], ga);
          for (int o = g >> 1; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o, g);
          double cs = 1.0, sn = 0.0;
          if (act) act = ga != 0.0 && ga * ga > tol2 * al * be && jacobi_rotation(al, be, ga, cs, sn);
          if (act) {
            double *gp = G + n * p, *gq = G + n * q, *vp = V + n * p, *vq = V + n * q;
            for (int i = li; i < n; i += g) {
              const double x = gp[i], y = gq[i];
              gp[i] = fma(-sn, y, cs * x);
              gq[i] = fma(sn, x, cs * y);
              const double xv = vp[i], yv = vq[i];
              vp[i] = fma(-sn, yv, cs * xv);
              vq[i] = fma(sn, xv, cs * yv);
            }
            if (li == 0) {
              const double c2 = cs * cs, s2 = sn * sn, cg = 2.0 * cs * sn * ga;
              nrm[p] = fma(c2, al, fma(s2, be, -cg));
              nrm[q] = fma(s2, al, fma(c2, be, cg));
              s_rot2 = 1;
            }
          }
        }
        __syncthreads();
      }
      const int rotated = s_rot2;
      __syncthreads();
      if (!rotated) break;
    }
  }
  // ---- singular values (column norms of G), order, truncation
  for (int j = warp; j < n; j += kSvdWarps) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s = fma(G[i + n * j], G[i + n * j], s);
    s = dwarp_sum(s);
    if (lane == 0) nrm[j] = sqrt(s);
  }
  __syncthreads();
  // s_order[rank] = column of G holding the rank-th largest singular value (stable)
  __shared__ int s_order[1024];
  for (int j = threadIdx.x; j < n; j += kSvdThreads) {
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
    const double delta2 = a.dm1 > 0 ? a.tol * a.tol * (*a.norm2) / (double)a.dm1 : 0.0;
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
    if (bad) set_status(a.status, TNR_ENONFINITE);
    if (a.max_rank > 0 && r > a.max_rank) r = (int)a.max_rank;
    if (r < 1) r = 1;
    s_r = (int)r;
    *a.r_out = (int64_t)r;
  }
  __syncthreads();
  const int r = s_r;
  // ---- outputs
  // left factor U_G[:, :r] diag(S) = G[:, order[:r]] (the Jacobi columns are U_G S), right
  // factor V[:, order[:r]]. One of them is mapped through Q_x: W (mm x r) = Q_x [Z; 0].
  // tall : Z = G[:, order[:r]] -> US = Q_x Z (t x r); core = V[:, order]^T (r x w)
  // wide : Z = V[:, order[:r]] -> core = (Q_x Z)^T (r x w); US = G[:, order] (t x r)
  for (int idx = threadIdx.x; idx < mm * r; idx += kSvdThreads) {
    const int i = idx % mm, c = idx / mm;
    const int col = s_order[c];
    W[idx] = i < n ? (tall ? G[i + n * col] : V[i + n * col]) : 0.0;
  }
  __syncthreads();
  for (int i = n - 1; i >= 0; --i) {  // W <- H_i W, i = n-1 .. 0
    const double tv = tau[i];
    if (tv == 0.0) continue;
    const double *v = X + mm * i;
    for (int c = warp; c < r; c += kSvdWarps) {
      double *col = W + mm * c;
      double s = lane == 0 ? col[i] : 0.0;
      for (int q = i + 1 + lane; q < mm; q += 32) s = fma(v[q], col[q], s);
      s = dwarp_sum(s) * tv;
      if (lane == 0) col[i] -= s;
      for (int q = i + 1 + lane; q < mm; q += 32) col[q] = fma(-s, v[q], col[q]);
    }
    __syncthreads();
  }
  if (tall) {
    for (int idx = threadIdx.x; idx < t * r; idx += kSvdThreads) a.US[idx] = W[idx];  // t x r, ld t = mm
    for (int idx = threadIdx.x; idx < r * w; idx += kSvdThreads) {
      const int c = idx % r, j = idx / r;
      a.core_out[idx] = V[j + n * s_order[c]];
    }
  } else {
    for (int idx = threadIdx.x; idx < r * w; idx += kSvdThreads) {
      const int c = idx % r, j = idx / r;
      a.core_out[idx] = W[j + mm * c];
    }
    for (int idx = threadIdx.x; idx < t * r; idx += kSvdThreads) {
      const int i = idx % t, c = idx / t;
      a.US[idx] = G[i + n * s_order[c]];
    }
  }
}

}  // namespace

size_t svd_step_smem(int64_t t, int64_t w) {
  const int64_t mm = t >= w ? t : w, n = t >= w ? w : t;
  return sizeof(double) * (2 * mm * n + 2 * n * n + 2 * n);
}

int svd_step_small(cudaStream_t s, const double *M, int64_t t, int64_t w, const double *norm2, double tol,
                   int64_t dm1, int64_t max_rank, double *core_out, double *US, int64_t *r_dev) {
  const size_t smem = svd_step_smem(t, w);
  const int64_t n = t < w ? t : w;
  if (smem > 200 * 1024 || n > 1024) return TNR_EINVAL;
  SvdStepArgs a{M, t, w, norm2, tol, dm1, max_rank, core_out, US, r_dev, status_ptr()};
  if (smem > 48 * 1024) TNR_CK(cudaFuncSetAttribute(k_svd_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LaunchScope ls(K_SVD, s);
  k_svd_step<<<1, kSvdThreads, smem, s>>>(a);
  return check_cuda(cudaGetLastError());
}

}  // namespace tnr
