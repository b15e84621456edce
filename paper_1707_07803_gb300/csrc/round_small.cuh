// The fused one-CTA rounding sweeps of Section 5.4 as device code (see round_small.cu), shared
// by the standalone kernel and the cooperative compression kernel, which runs them right after
// the compression when the cores fit its shared memory.
#pragma once

#include "cta_linalg.cuh"

namespace tnr {

struct RoundSmallArgs {
  int d;
  double *core[TNR_MAX_SITES];
  int phys[TNR_MAX_SITES];   // I_k J_k (row multiplicity of core k)
  int R[TNR_MAX_SITES + 1];  // ranks on entry
  int off[TNR_MAX_SITES];    // shared-memory offset of core k (doubles)
  int tmp_off, tmp_cap, rbuf_off, work_off, gram_off;
  int certify;  // cores 1..d-1 are right-orthonormal on entry: try the no-truncation certificate
  // G_1 = C_0^T C_0 as g1_parts partial Grams (R[1] x R[1] each, global memory, R[1] <= 16) to be
  // added in order, when the caller spread it over a grid; null: the CTA forms G_1 itself
  const double *g1_part;
  int g1_parts;
  double tol;
  int64_t max_rank;
  int64_t *R_out;  // device, d + 1 ranks on exit
  int *status;
};

// No-truncation certificate for the rounding (Section 5.4), valid when cores 1..d-1 are
// right-orthonormal (as the exact right-to-left compression leaves them). Then the singular
// values at bond k are those of the left part Y_{<k}, whose Gram matrix follows the recurrence
// G_1 = C_0^T C_0, G_{k+1} = sum_{a, a', x} C_k(a, x, .) G_k(a, a') C_k(a', x, .), and
// ||Y||_F^2 = trace(G_1). If every bond keeps sigma_min^2 >= 1 / trace(G_k^{-1}) > delta^2 and
// no rank exceeds max_rank, both sweeps would keep every singular value and only change the
// gauge: the rounded tensor is Y itself. A bound that is off by rounding can only keep a
// component smaller than delta, the truncation error the rounding allows anyway.
// Returns 1 (uniform over the CTA) when certified.
static __device__ int bonds_certified(const RoundSmallArgs &a, const double *sm, const int *Rs, double *tmp, double *gram,
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (a.g1_part && Rs[1] <= 16) {
    // G_1 from the grid's partials: thread (entry e, stripe s) adds partials s, s + S, ... (all its
    // loads in flight), then the S stripe sums of each entry are added in order
    __shared__ double red[kStepThreads];
    const int r1 = Rs[1], E2 = r1 * r1, S = kStepThreads / E2, e = threadIdx.x % E2, st = threadIdx.x / E2;
    double v = 0.0;
    if (st < S)
#pragma unroll 4
      for (int b = st; b < a.g1_parts; b += S) v += __ldcg(a.g1_part + (int64_t)b * E2 + e);
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < E2) {
      double s0 = 0.0;
      for (int q = 0; q < S; ++q) s0 += red[threadIdx.x + q * E2];
      gram[goff[1] + threadIdx.x] = s0;
    }
    __syncthreads();
  } else {
    cta_tn_sym(gram + goff[1], sm + a.off[0], sm + a.off[0], Rs[0] * a.phys[0], Rs[1]);
  }
  for (int k = 1; k + 1 < d; ++k) {
    const int r = Rs[k], ph = a.phys[k], r2 = Rs[k + 1], w = ph * r2;
    const double *C = sm + a.off[k], *G = gram + goff[k];
    if (r <= 8 && r * ph * r2 <= a.tmp_cap) {
      // small bond, two short phases over the whole CTA: T = G_k C_k (r x (ph r'), one output per
      // thread, an r-term chain), then G_{k+1}(b, b') = sum_{(a, x)} C((a, x), b) T((a, x), b') for
      // b <= b' by groups of eight lanes (three-level shuffle sum): the chain per site is ~r + 6
      // dependent FP64 operations instead of a per-entry product and a five-level warp sum
      double *Gn = gram + goff[k + 1];
      const int m = r * ph, nT = m * r2, E = r2 * (r2 + 1) / 2;
      for (int idx = threadIdx.x; idx < nT; idx += kStepThreads) {
        const int aa = idx % r, col = idx / r;
        const double *cc = C + r * col;
        double t = 0.0;
        for (int a2 = 0; a2 < r; ++a2) t = fma(G[aa + r * a2], cc[a2], t);
        tmp[idx] = t;
      }
      __syncthreads();
      const int part = threadIdx.x & 7, ngroups = kStepThreads / 8;
      // g0: the warp's first group, so the loop condition (and the shuffles) are warp-uniform
      for (int ee = threadIdx.x >> 3, g0 = warp * 4; g0 < E; ee += ngroups, g0 += ngroups) {
        int j = 0, base = 0;
        const bool live = ee < E;
        if (live)
          while (base + j + 1 <= ee) {
            base += j + 1;
            ++j;
          }
        const int i = ee - base;  // (i, j) = (b, b'), i <= j
        double sacc = 0.0;
        if (live) {
          const double *ci = C + m * i, *tj = tmp + m * j;
          for (int ax = part; ax < m; ax += 8) sacc = fma(ci[ax], tj[ax], sacc);
        }
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 4);
        if (live && part == 0) {
          Gn[i + r2 * j] = sacc;
          Gn[j + r2 * i] = sacc;
        }
      }
      __syncthreads();
    } else {
      cta_gemm(tmp, G, r, C, r, r, w, r);  // T = G_k C_k (r x phys r')
      cta_tn_sym(gram + goff[k + 1], C, tmp, r * ph, r2);
    }
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < Rs[1]; ++b) t += gram[goff[1] + b + Rs[1] * b];
    sc[0] = a.tol * a.tol * t / (double)(d - 1);  // delta^2
  }
  __syncthreads();
  const double delta2 = sc[0];
  // one warp per bond
  for (int k = 1 + warp; k < d; k += kStepWarps) {
    const double lb = warp_lambda_min_bound(gram + goff[k], Rs[k]);
    if (lane == 0 && !(lb > delta2 * (1.0 + 1e-6))) atomicExch(&s_ok, 0);
  }
  __syncthreads();
  return s_ok;
}

// Both sweeps (or the certificate) for the cores of `a`, by the whole calling CTA (kStepThreads
// threads) with `sm` as the shared-memory area laid out by round_small_layout.
static __device__ __noinline__ void round_small_body(const RoundSmallArgs &a, double *sm) {
  __shared__ int Rs[TNR_MAX_SITES + 1];
  __shared__ double red[8 * kStepWarps];
  __shared__ double sc[8];
  const int d = a.d;
  for (int k = threadIdx.x; k <= d; k += kStepThreads) Rs[k] = a.R[k];
  // the certificate with G_1 from the grid's partials never reads core 0: it is loaded only when
  // the sweeps have to run
  const bool lazy0 = a.certify && a.g1_part && a.R[1] <= 16;
  // every core's loads in flight together: one pass over the concatenated index range, four
  // elements per thread loaded before any is stored (through L2: inside the cooperative
  // compression other CTAs wrote these cores)
  {
    const int k0 = lazy0 ? 1 : 0;
    int total = 0;
    for (int k = k0; k < d; ++k) total += a.R[k] * a.phys[k] * a.R[k + 1];
    for (int g0 = threadIdx.x; g0 < total; g0 += 4 * kStepThreads) {
      double v[4];
      int dst[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int g = g0 + u * kStepThreads;
        dst[u] = -1;
        if (g < total) {
          int k = k0, n = a.R[k] * a.phys[k] * a.R[k + 1];
          while (g >= n) {
            g -= n;
            ++k;
            n = a.R[k] * a.phys[k] * a.R[k + 1];
          }
          dst[u] = a.off[k] + g;
          v[u] = __ldcg(a.core[k] + g);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u] >= 0) sm[dst[u]] = v[u];
    }
  }
  __syncthreads();
  double *tmp = sm + a.tmp_off, *rbuf = sm + a.rbuf_off, *work = sm + a.work_off;
  if (a.certify && bonds_certified(a, sm, Rs, tmp, sm + a.gram_off, sc)) {
    for (int k = threadIdx.x; k <= d; k += kStepThreads) a.R_out[k] = Rs[k];  // cores unchanged
    return;
  }
  if (lazy0) {
    const int n = a.R[0] * a.phys[0] * a.R[1];
    for (int i = threadIdx.x; i < n; i += kStepThreads) sm[a.off[0] + i] = __ldcg(a.core[0] + i);
    __syncthreads();
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

// Shared-memory bytes of the fused sweeps for cores with ranks R (d + 1) and row multiplicities
// phys (I_k J_k); 0 when some dimension is out of range.
static __host__ __device__ size_t round_small_layout(const int64_t *R, const int64_t *phys, int d,
                                                     RoundSmallLayout *lay) {
  if (d < 2 || d > TNR_MAX_SITES) return 0;
  int64_t off = 0, maxcore_tail = 1, maxbond = 1, maxwork = 1, gram = 0;
  for (int k = 0; k < d; ++k) {
    const int64_t ph = phys[k];
    if (ph <= 0 || ph > (1 << 20) || R[k] > kStepMaxN || R[k + 1] > kStepMaxN) return 0;
    const int64_t n = R[k] * ph * R[k + 1];
    if (n > (1 << 22)) return 0;
    lay->off[k] = (int)off;
    off += (n + 3) & ~int64_t(3);  // 32-byte aligned regions
    if (k >= 1) {
      maxcore_tail = maxcore_tail > n ? maxcore_tail : n;
      const int64_t t = R[k], w = ph * R[k + 1];
      if ((t < w ? t : w) > kStepMaxN) return 0;
      const int64_t sw = svd_step_work(t, w);
      maxwork = maxwork > sw ? maxwork : sw;
    }
    const int64_t mb = R[k] > R[k + 1] ? R[k] : R[k + 1];
    maxbond = maxbond > mb ? maxbond : mb;
    if (k >= 1) gram += R[k] * R[k];
  }
  // tmp: output of the L->R absorb (at most a core of site >= 1) and the row blocks of the
  // R->L absorb (at least one row of maxbond values)
  const int64_t tmp_cap = maxcore_tail > 32 * maxbond ? maxcore_tail : 32 * maxbond;
  lay->tmp_off = (int)off;
  lay->tmp_cap = (int)tmp_cap;
  off += (tmp_cap + 3) & ~int64_t(3);
  lay->rbuf_off = (int)off;  // R factors (nq x cols) and U S (t x r): at most maxbond^2
  off += (maxbond * maxbond + 3) & ~int64_t(3);
  lay->work_off = (int)off;  // SVD-step workspace, or the QR's tau (at most maxbond)
  off += ((maxwork > maxbond ? maxwork : maxbond) + 3) & ~int64_t(3);
  lay->gram_off = (int)off;  // Gram matrices of bonds 1..d-1 for the certificate
  off += gram;
  return sizeof(double) * (size_t)off;
}

// Fills the kernel arguments for cores `core` with ranks R and multiplicities phys.
static __host__ __device__ void round_small_args(RoundSmallArgs &a, const RoundSmallLayout &lay, int d,
                                                 double *const *core, const int64_t *R, const int64_t *phys,
                                                 bool certify, double tol, int64_t max_rank, int64_t *R_out,
                                                 int *status) {
  a.d = d;
  for (int k = 0; k < d; ++k) {
    a.core[k] = core[k];
    a.phys[k] = (int)phys[k];
    a.off[k] = lay.off[k];
  }
  for (int k = 0; k <= d; ++k) a.R[k] = (int)R[k];
  a.tmp_off = lay.tmp_off;
  a.tmp_cap = lay.tmp_cap;
  a.rbuf_off = lay.rbuf_off;
  a.work_off = lay.work_off;
  a.gram_off = lay.gram_off;
  a.certify = certify ? 1 : 0;
  a.g1_part = nullptr;
  a.g1_parts = 0;
  a.tol = tol;
  a.max_rank = max_rank;
  a.R_out = R_out;
  a.status = status;
}

}  // namespace tnr
