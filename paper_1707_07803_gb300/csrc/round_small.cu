// Fused rounding sweeps for MPOs whose cores all fit in one CTA's shared memory.
//
// Section 5.4 integrates SVD-based rounding with the MPO-QR of Alg. 5.2: a left-to-right QR
// sweep (core k reshaped (R_k I_k J_k) x R_{k+1} = Q R, R absorbed into core k+1) followed by a
// right-to-left sweep that, per core, takes the truncated SVD of R_k x (I_k J_k R_{k+1}), keeps
// V^T as the new (right-orthogonal) core and absorbs U S into core k-1. When every core fits in
// shared memory the whole sequence is one launch: the cores are read once and written once, the
// ranks stay on the device, and each step's small dense factorisation is a device function run
// by the whole CTA, so there is no launch, host round trip or global-memory staging per bond.
// The site-1 step of Alg. 5.2/5.3 follows separately.
#include "svd_step.cuh"

namespace tnr {
namespace {

struct RoundSmallArgs {
  int d;
  double *core[TNR_MAX_SITES];
  int phys[TNR_MAX_SITES];   // I_k J_k (row multiplicity of core k)
  int R[TNR_MAX_SITES + 1];  // ranks on entry
  int off[TNR_MAX_SITES];    // shared-memory offset of core k (doubles)
  int tmp_off, tmp_cap, rbuf_off, work_off, gram_off;
  int certify;  // cores 1..d-1 are right-orthonormal on entry: try the no-truncation certificate
  double tol;
  int64_t max_rank;
  int64_t *R_out;  // device, d + 1 ranks on exit
  int *status;
};

// GB300 issues FP64 at 1/64 of the FP32 rate: one FP64 warp instruction holds a sub-partition's
// FP64 pipe for ~70 cycles whether 1 or 32 lanes are active. The helpers below therefore keep the
// FP64 instruction count per CTA close to the arithmetic itself: partial sums are reduced only by
// warps that own rows, scalar work (final sums, reflector parameters) is done once by one thread
// or lane-parallel in one warp, and results are broadcast through shared memory.

// Number of warps owning at least one of `rows` rows when row r goes to thread r % kStepThreads.
__device__ __forceinline__ int active_warps(int rows) {
  const int w = (rows + 31) >> 5;
  return w < kStepWarps ? w : kStepWarps;
}

// Sum over the CTA of per-thread values of the first `rows` threads' strided rows; the total is
// returned to every thread. red: kStepWarps doubles.
__device__ __forceinline__ double cta_sum(double v, int rows, double *red, double *out) {
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
__device__ void cta_reflect(const double *v, int i, int m, double tau, double *A, int lda, int j0, int j1,
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
__device__ void cta_qr(double *A, int m, int n, double *Rout, double *tau, double *red, double *sc) {
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
__device__ void cta_gemm(double *C, const double *A, int lda, const double *B, int ldb, int m, int n, int k) {
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
__device__ void cta_absorb_right(double *C, int rows, int t, const double *US, int r, double *tmp, int cap) {
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
__device__ void cta_tn_sym(double *G, const double *A, const double *B, int m, int r) {
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
__device__ double warp_lambda_min_bound(double *G, int r) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int j = 0; j < r; ++j) {
    const double dj = G[j + r * j];
    if (!(dj > 0.0) || !isfinite(dj)) {
      ok = false;
      break;
    }
    const double inv = 1.0 / dj;  // one division sequence per pivot (lane-uniform)
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

// No-truncation certificate for the rounding (Section 5.4), valid when cores 1..d-1 are
// right-orthonormal (as the exact right-to-left compression leaves them). Then the singular
// values at bond k are those of the left part Y_{<k}, whose Gram matrix follows the recurrence
// G_1 = C_0^T C_0, G_{k+1} = sum_{a, a', x} C_k(a, x, .) G_k(a, a') C_k(a', x, .), and
// ||Y||_F^2 = trace(G_1). If every bond keeps sigma_min^2 >= 1 / trace(G_k^{-1}) > delta^2 and
// no rank exceeds max_rank, both sweeps would keep every singular value and only change the
// gauge: the rounded tensor is Y itself. A bound that is off by rounding can only keep a
// component smaller than delta, the truncation error the rounding allows anyway.
// Returns 1 (uniform over the CTA) when certified.
__device__ int bonds_certified(const RoundSmallArgs &a, const double *sm, const int *Rs, double *tmp, double *gram,
                               double *sc) {
  __shared__ int goff[TNR_MAX_SITES];
  __shared__ int s_ok;
  const int d = a.d;
  if (threadIdx.x == 0) {
    int off = 0;
    int ok = 1;
    for (int k = 1; k < d; ++k) {
      goff[k] = off;
      off += Rs[k] * Rs[k];
      if (Rs[k] > 32 || (a.max_rank > 0 && Rs[k] > a.max_rank)) ok = 0;
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return 0;
  // Gram chain
  cta_tn_sym(gram + goff[1], sm + a.off[0], sm + a.off[0], Rs[0] * a.phys[0], Rs[1]);
  for (int k = 1; k + 1 < d; ++k) {
    const int r = Rs[k], w = a.phys[k] * Rs[k + 1];
    cta_gemm(tmp, gram + goff[k], r, sm + a.off[k], r, r, w, r);  // T = G_k C_k (r x phys r')
    cta_tn_sym(gram + goff[k + 1], sm + a.off[k], tmp, r * a.phys[k], Rs[k + 1]);
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < Rs[1]; ++b) t += gram[goff[1] + b + Rs[1] * b];
    sc[0] = a.tol * a.tol * t / (double)(d - 1);  // delta^2
  }
  __syncthreads();
  const double delta2 = sc[0];
  // one warp per bond
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 1 + warp; k < d; k += kStepWarps) {
    const double lb = warp_lambda_min_bound(gram + goff[k], Rs[k]);
    if (lane == 0 && !(lb > delta2 * (1.0 + 1e-6))) atomicExch(&s_ok, 0);
  }
  __syncthreads();
  return s_ok;
}

__global__ void __launch_bounds__(kStepThreads) k_round_small(RoundSmallArgs a) {
  extern __shared__ double sm[];
  __shared__ int Rs[TNR_MAX_SITES + 1];
  __shared__ double red[8 * kStepWarps];
  __shared__ double sc[8];
  const int d = a.d;
  for (int k = threadIdx.x; k <= d; k += kStepThreads) Rs[k] = a.R[k];
  for (int k = 0; k < d; ++k) {
    const int n = a.R[k] * a.phys[k] * a.R[k + 1];
    const double *src = a.core[k];
    double *dst = sm + a.off[k];
    for (int i = threadIdx.x; i < n; i += kStepThreads) dst[i] = src[i];
  }
  __syncthreads();
  double *tmp = sm + a.tmp_off, *rbuf = sm + a.rbuf_off, *work = sm + a.work_off;
  if (a.certify && bonds_certified(a, sm, Rs, tmp, sm + a.gram_off, sc)) {
    for (int k = threadIdx.x; k <= d; k += kStepThreads) a.R_out[k] = Rs[k];  // cores unchanged
    return;
  }
  // left-to-right QR sweep: core k = Q R, R absorbed into core k+1
  for (int k = 0; k + 1 < d; ++k) {
    const int rows = Rs[k] * a.phys[k], cols = Rs[k + 1];
    const int nq = rows < cols ? rows : cols;
    cta_qr(sm + a.off[k], rows, cols, rbuf, work, red, sc);
    const int w = a.phys[k + 1] * Rs[k + 2];
    cta_gemm(tmp, rbuf, nq, sm + a.off[k + 1], cols, nq, w, cols);
    for (int i = threadIdx.x; i < nq * w; i += kStepThreads) sm[a.off[k + 1] + i] = tmp[i];
    if (threadIdx.x == 0) Rs[k + 1] = nq;
    __syncthreads();
  }
  // ||Y||_F^2 = ||last core||_F^2 (all other cores are left-orthogonal now)
  double nrm2;
  {
    const int n = Rs[d - 1] * a.phys[d - 1] * Rs[d];
    const double *c = sm + a.off[d - 1];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kStepThreads) s = fma(c[i], c[i], s);
    nrm2 = cta_sum(s, n, red, sc);
  }
  const double delta2 = a.tol * a.tol * nrm2 / (double)(d - 1);
  // right-to-left truncating sweep: core k = (U S) V^T, V^T kept, U S absorbed into core k-1
  for (int k = d - 1; k >= 1; --k) {
    const int t = Rs[k], w = a.phys[k] * Rs[k + 1];
    const int r = svd_step_cta(sm + a.off[k], t, w, delta2, a.max_rank, sm + a.off[k], rbuf, work, a.status);
    cta_absorb_right(sm + a.off[k - 1], Rs[k - 1] * a.phys[k - 1], t, rbuf, r, tmp, a.tmp_cap);
    if (threadIdx.x == 0) Rs[k] = r;
    __syncthreads();
  }
  for (int k = 0; k < d; ++k) {
    const int n = Rs[k] * a.phys[k] * Rs[k + 1];
    const double *src = sm + a.off[k];
    double *dst = a.core[k];
    for (int i = threadIdx.x; i < n; i += kStepThreads) dst[i] = src[i];
  }
  for (int k = threadIdx.x; k <= d; k += kStepThreads) a.R_out[k] = Rs[k];
}

struct RoundSmallLayout {
  int off[TNR_MAX_SITES];
  int tmp_off, tmp_cap, rbuf_off, work_off, gram_off;
};

// Shared-memory bytes for the fused sweeps on Y (0 when some dimension is out of range).
size_t round_small_layout(const tnr_mpo &Y, RoundSmallLayout *lay) {
  const int d = Y.d;
  if (d < 2 || d > TNR_MAX_SITES) return 0;
  int64_t off = 0, maxcore_tail = 1, maxbond = 1, maxwork = 1, gram = 0;
  for (int k = 0; k < d; ++k) {
    const int64_t phys = Y.I[k] * Y.J[k];
    if (phys <= 0 || phys > (1 << 20) || Y.R[k] > kStepMaxN || Y.R[k + 1] > kStepMaxN) return 0;
    const int64_t n = Y.R[k] * phys * Y.R[k + 1];
    if (n > (1 << 22)) return 0;
    lay->off[k] = (int)off;
    off += (n + 3) & ~int64_t(3);  // 32-byte aligned regions
    if (k >= 1) {
      maxcore_tail = std::max(maxcore_tail, n);
      const int64_t t = Y.R[k], w = phys * Y.R[k + 1];
      if (std::min(t, w) > kStepMaxN) return 0;
      maxwork = std::max(maxwork, svd_step_work(t, w));
    }
    maxbond = std::max(maxbond, std::max(Y.R[k], Y.R[k + 1]));
    if (k >= 1) gram += Y.R[k] * Y.R[k];
  }
  // tmp: output of the L->R absorb (at most a core of site >= 1) and the row blocks of the
  // R->L absorb (at least one row of maxbond values)
  const int64_t tmp_cap = std::max(maxcore_tail, 32 * maxbond);
  lay->tmp_off = (int)off;
  lay->tmp_cap = (int)tmp_cap;
  off += (tmp_cap + 3) & ~int64_t(3);
  lay->rbuf_off = (int)off;  // R factors (nq x cols) and U S (t x r): at most maxbond^2
  off += (maxbond * maxbond + 3) & ~int64_t(3);
  lay->work_off = (int)off;  // SVD-step workspace, or the QR's tau (at most maxbond)
  off += (std::max(maxwork, maxbond) + 3) & ~int64_t(3);
  lay->gram_off = (int)off;  // Gram matrices of bonds 1..d-1 for the certificate
  off += gram;
  return sizeof(double) * (size_t)off;
}

}  // namespace

// Runs both rounding sweeps of Y in one launch when they fit one CTA's shared memory; otherwise
// launches nothing and leaves *launched false. Ranks on exit go to R_dev (d + 1 values).
// certify: cores 1..d-1 are right-orthonormal, so the no-truncation certificate may skip the sweeps.
int round_small(cudaStream_t s, const tnr_mpo &Y, double tol, int64_t max_rank, bool certify, int64_t *R_dev,
                bool *launched) {
  *launched = false;
  RoundSmallLayout lay;
  const size_t smem = round_small_layout(Y, &lay);
  if (smem == 0 || smem > kRoundSmallMaxSmem) return TNR_OK;
  RoundSmallArgs a;
  a.d = Y.d;
  for (int k = 0; k < Y.d; ++k) {
    a.core[k] = Y.core[k];
    a.phys[k] = (int)(Y.I[k] * Y.J[k]);
    a.off[k] = lay.off[k];
  }
  for (int k = 0; k <= Y.d; ++k) a.R[k] = (int)Y.R[k];
  a.tmp_off = lay.tmp_off;
  a.tmp_cap = lay.tmp_cap;
  a.rbuf_off = lay.rbuf_off;
  a.work_off = lay.work_off;
  a.gram_off = lay.gram_off;
  a.certify = certify ? 1 : 0;
  a.tol = tol;
  a.max_rank = max_rank;
  a.R_out = R_dev;
  a.status = status_ptr();
  TNR_TRY(ensure_dynamic_smem((const void *)k_round_small, smem));
  {
    LaunchScope ls(K_ROUND, s);
    k_round_small<<<1, kStepThreads, smem, s>>>(a);
  }
  TNR_CK(cudaGetLastError());
  *launched = true;
  return TNR_OK;
}

}  // namespace tnr
