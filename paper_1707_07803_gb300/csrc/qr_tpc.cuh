// One-CTA Householder QR of a short matrix (m <= 64 rows), one thread per column, with optional
// column pivoting and a cutoff: the body of k_qr_small_tpc as a device function, so that other
// kernels (the device-side compression sweep) can run it on their own data. All kSmallThreads
// threads of the CTA call it.
#pragma once

#include "dev_common.cuh"
#include "tnr_internal.cuh"

namespace tnr {

constexpr int kSmallThreads = 256;

// Bytes of the shared-memory layout of qr_tpc_cta for an m x n matrix.
__host__ __device__ inline int64_t qr_tpc_bytes(int64_t m, int64_t n) {
  return (int64_t)sizeof(double) * (m * n + 2 * n + (m < n ? m : n) + m) + (int64_t)sizeof(int) * n;
}

struct QrSmallArgs {
  const double *src;
  int64_t lds;
  int64_t m, n;
  int trans_src, pivot, trans_q, trans_r;
  double cut_rel;
  double *Q;
  int64_t ldq;
  double *R;
  int64_t ldr;
  int64_t *r_out;
};

// One thread owns one column and streams it alone, so no FP64 shuffle reductions are spent on
// columns shorter than a warp; the matrix is kept row-major in shared memory (consecutive threads
// touch consecutive words). Column pivoting uses norm downdating with the LAPACK (dgeqp3)
// safeguard: the norm of column j below row i is updated as ||.||^2 - R(i,j)^2 and recomputed
// when the downdate has lost more than half of its digits. Outputs as k_qr_small: Q (m x r) as Q
// or Q^T (ldq <= 0 packs Q^T with leading dimension r), R = Q^T A (r x n, original column order)
// as R or R^T, r to *r_out. Shared memory: m n + 2 n + min(m, n) + m doubles and n ints.
static __device__ __noinline__ void qr_tpc_cta(const QrSmallArgs &a, double *sm) {
  const int m = a.m, n = a.n;
  const int nref = m < n ? m : n;
  double *A = sm;                 // m x n row-major: A(t, j) at t * n + j
  double *nrm = A + m * n;        // n: current squared norms below the active row
  double *nrm0 = nrm + n;         // n: squared norms at the last recompute
  double *tau = nrm0 + n;         // nref
  double *vv = tau + nref;        // m: current reflector
  int *perm = reinterpret_cast<int *>(vv + m);  // n
  __shared__ double s_red[32];
  __shared__ int s_idx[32];
  __shared__ long long s_key[32];
  __shared__ int s_r;
  __shared__ double s_cut2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kSmallThreads / 32;
  for (int idx = threadIdx.x; idx < m * n; idx += kSmallThreads) {
    const int j = idx % n, t = idx / n;
    // read through L2: the source may have been written by other CTAs of a cooperative kernel
    A[idx] = __ldcg(a.trans_src ? a.src + (j + a.lds * t) : a.src + (t + a.lds * j));
  }
  __syncthreads();
  double fro = 0.0;
  for (int j = threadIdx.x; j < n; j += kSmallThreads) {
    double s = 0.0;
    for (int t = 0; t < m; ++t) s = fma(A[t * n + j], A[t * n + j], s);
    nrm[j] = s;
    nrm0[j] = s;
    perm[j] = (int)j;
    fro += s;
  }
  fro = dwarp_sum(fro);
  if (lane == 0) s_red[warp] = fro;
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int w = 0; w < NW; ++w) f += s_red[w];
    s_cut2 = a.cut_rel * a.cut_rel * f;
    s_r = (int)nref;
  }
  __syncthreads();
  for (int i = 0; i < nref; ++i) {
    if (a.pivot) {
      // argmax of the remaining column norms; the norms are >= 0, so their bit patterns order
      // like the values and the comparisons stay on the integer pipe (ties: lowest index)
      long long bv = -1;
      int bi = (int)i;
      for (int j = i + threadIdx.x; j < n; j += kSmallThreads) {
        const long long v = __double_as_longlong(nrm[j]);
        if (v > bv) {
          bv = v;
          bi = (int)j;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_key[warp] = bv;
        s_idx[warp] = bi;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        long long b = s_key[0];
        int bj = s_idx[0];
        for (int w = 1; w < NW; ++w)
          if (s_key[w] > b || (s_key[w] == b && s_idx[w] < bj)) {
            b = s_key[w];
            bj = s_idx[w];
          }
        s_idx[0] = bj;
        if (i > 0 && __longlong_as_double(b) <= s_cut2) s_r = (int)i;
      }
      __syncthreads();
      if (s_r == (int)i) break;
      const int p = s_idx[0];
      if (p != i) {
        for (int t = threadIdx.x; t < m; t += kSmallThreads) {
          const double x = A[t * n + i];
          A[t * n + i] = A[t * n + p];
          A[t * n + p] = x;
        }
        if (threadIdx.x == 0) {
          double x = nrm[i];
          nrm[i] = nrm[p];
          nrm[p] = x;
          x = nrm0[i];
          nrm0[i] = nrm0[p];
          nrm0[p] = x;
          const int q = perm[i];
          perm[i] = perm[p];
          perm[p] = q;
        }
      }
      __syncthreads();
    }
    if (warp == 0) {  // reflector from column i, rows i..m-1
      double sig = 0.0;
      for (int t = i + 1 + lane; t < m; t += 32) sig = fma(A[t * n + i], A[t * n + i], sig);
      sig = dwarp_sum(sig);
      const double alpha = A[i * n + i];
      double tv = 0.0, beta = alpha, scal = 0.0;
      if (sig > 0.0) {
        householder_params(alpha, sig, beta, tv, scal);
      }
      for (int t = i + 1 + lane; t < m; t += 32) {
        const double x = A[t * n + i] * scal;
        A[t * n + i] = x;
        vv[t] = x;
      }
      __syncwarp();
      if (lane == 0) {
        A[i * n + i] = beta;
        tau[i] = tv;
        vv[i] = 1.0;
      }
    }
    __syncthreads();
    const double tv = tau[i];
    for (int j = i + 1 + threadIdx.x; j < n; j += kSmallThreads) {
      if (tv != 0.0) {
        double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        int t = i;
        for (; t + 3 < m; t += 4) {
          w0 = fma(vv[t], A[t * n + j], w0);
          w1 = fma(vv[t + 1], A[(t + 1) * n + j], w1);
          w2 = fma(vv[t + 2], A[(t + 2) * n + j], w2);
          w3 = fma(vv[t + 3], A[(t + 3) * n + j], w3);
        }
        for (; t < m; ++t) w0 = fma(vv[t], A[t * n + j], w0);
        const double w = ((w0 + w1) + (w2 + w3)) * tv;
        for (t = i; t < m; ++t) A[t * n + j] = fma(-w, vv[t], A[t * n + j]);
      }
      if (a.pivot) {
        const double rij = A[i * n + j];
        double nn = nrm[j] - rij * rij;
        // dgeqp3 safeguard: recompute once the downdate has cancelled too much
        if (nn <= 1.4901161193847656e-08 * nrm0[j] || nn < 0.0) {
          nn = 0.0;
          for (int t = i + 1; t < m; ++t) nn = fma(A[t * n + j], A[t * n + j], nn);
          nrm0[j] = nn;
        }
        nrm[j] = nn;
      }
    }
    __syncthreads();
  }
  const int r = s_r;
  if (threadIdx.x == 0 && a.r_out) *a.r_out = r;
  const int ldq = a.ldq > 0 ? a.ldq : r;
  for (int idx = threadIdx.x; idx < r * n; idx += kSmallThreads) {
    const int t = idx % r, j = idx / r;
    const double x = t <= j ? A[t * n + j] : 0.0;
    const int oj = perm[j];
    if (a.trans_r)
      a.R[oj + a.ldr * t] = x;
    else
      a.R[t + a.ldr * oj] = x;
  }
  // Q = H_0 ... H_{r-1} [I_r; 0]: warp w builds columns l = w, w + NW, ... with lanes over the
  // rows (two rows per lane, m <= 64); column l needs reflectors l .. 0 (backward accumulation)
  for (int l = warp; l < r; l += NW) {
    const int t0 = lane, t1 = lane + 32;
    double q0 = t0 == l ? 1.0 : 0.0, q1 = t1 == l ? 1.0 : 0.0;
    for (int j = l; j >= 0; --j) {
      const double tj = tau[j];
      if (tj == 0.0) continue;
      // v_j: 1 at row j, A(t, j) below, 0 above
      const double v0 = t0 < j || t0 >= m ? 0.0 : (t0 == j ? 1.0 : A[t0 * n + j]);
      const double v1 = t1 < j || t1 >= m ? 0.0 : (t1 == j ? 1.0 : A[t1 * n + j]);
      const double w = dwarp_sum(fma(v0, q0, v1 * q1)) * tj;
      q0 = fma(-w, v0, q0);
      q1 = fma(-w, v1, q1);
    }
    if (a.trans_q) {
      if (t0 < m) a.Q[l + ldq * t0] = q0;
      if (t1 < m) a.Q[l + ldq * t1] = q1;
    } else {
      if (t0 < m) a.Q[t0 + ldq * l] = q0;
      if (t1 < m) a.Q[t1 + ldq * l] = q1;
    }
  }
}

}  // namespace tnr
