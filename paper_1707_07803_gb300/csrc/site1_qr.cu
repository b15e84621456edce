// Site-1 QR of Algs. 5.2/5.3 (A1^T = Q~ R~, the (I1 t) x K matrix of the site-1 core) by
// CholeskyQR2 in ONE cooperative launch.
//
// Each CTA owns a block of rows of A1^T and keeps it in shared memory for both passes; a pass is
// a symmetric partial Gram per CTA, a fixed-order sum of the partials and the Cholesky factor on
// CTA 0, and the triangular solve of every CTA's rows (warp per row). Two bounded grid barriers
// per pass replace the six launches and the host round trip of the multi-kernel version, and the
// fixed-order sum makes the result independent of scheduling (no floating-point atomics).
//
// Pass 1 factors G1 = Y^T Y in the square-root-free form (one reciprocal per pivot). Pass 2 sees
// G2 = I + E with |E| ~ cond(Y)^2 eps; it first checks that G2 is within 0.5 / K of the identity
// (the regime in which CholeskyQR2 is orthogonal to rounding level; otherwise *flag is set and
// the caller falls back to Householder), and when max |E| <= 1e-9 its factor is taken in closed
// form, R2 = I + triu(E) - diag(E) / 2, whose error R2^T R2 - G2 = O(|E|^2) is below rounding
// level: no pivot chain at all. The result is R = R2 R1 and Q = Y R1^{-1} R2^{-1}.
#include <algorithm>

#include "dev_common.cuh"
#include "grid_sync.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

constexpr int kS1Threads = 256;
constexpr int kS1MaxK = 32;
constexpr int kS1MaxRowsPerCta = 384;

struct Site1Args {
  double *core0;          // (1, I1, K, t)
  const int64_t *t_dev;   // t in device memory (rank left there by the rounding), or null
  int I1, K, t;           // t: the rank when t_dev is null, else its upper bound
  int core_out;           // write Q~ back into core0's layout instead of Qout
  const int *gate;        // when not null and 0 on the device: do nothing (an earlier step declined)
  double *Gpart;        // gridDim.x partial Grams, K x K each
  double *S, *rdiag;    // the current pass's factor scaled to unit diagonal, and 1 / its diagonal
  double *Rout;         // K x K: R = R2 R1 (column-major, upper)
  double *Qout;         // m x K, column-major
  int *flag;            // set when the factorisation cannot be trusted
  unsigned *bar;
  int *status;
};

// 1 / x for finite x > 0 with one Newton step from the FP32 reciprocal (relative error ~2^-46): the
// pass-1 pivots only have to precondition, since Y = Q1 R1 holds exactly for the R1 the solve uses.
__device__ __forceinline__ double rcp_f64_1(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
  const double xs = x * pow2(-e);
  double q = (double)(1.0f / (float)xs);
  q = q * fma(-xs, q, 2.0);
  return q * pow2(-e);
}

// Cholesky of the K x K matrix a (shared, column-major, K <= 32) on one CTA of kS1Threads
// threads: R (upper) to Rs and 1 / diag(R) to rd (both shared; Rs must not alias a). Thread
// (lane, warp) owns the elements (i = lane, l = warp + 8 u), so no index division is needed.
// second: the CholeskyQR2 near-identity check and closed-form factor. Returns false (uniform
// over the CTA) when the factor cannot be used.
__device__ bool cta_chol(double *a, int K, double *Rs, double *rd, bool second, double *dinv) {
  __shared__ int s_bad, s_first;
  const int i = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kW = kS1Threads / 32;
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_first = 1;
  }
  __syncthreads();
  if (second) {
    bool bad = false, far = false;
    if (i < K)
      for (int l = w; l < K; l += kW) {
        const double dev = fabs(a[i + K * l] - (i == l ? 1.0 : 0.0));
        bad |= !(dev <= 0.5 / K);
        far |= !(dev <= 1e-9);
      }
    const bool wbad = __any_sync(0xffffffffu, bad), wfar = __any_sync(0xffffffffu, far);
    if (i == 0 && wbad) s_bad = 1;  // benign races: every writer stores the same value
    if (i == 0 && wfar) s_first = 0;
    __syncthreads();
    if (s_bad) return false;
    if (s_first) {  // G = I + E, R = I + triu(E) - diag(E) / 2 up to O(|E|^2)
      if (i < K)
        for (int l = w; l < K; l += kW) {
          const double v = i < l ? a[i + K * l] : (i == l ? 0.5 * (1.0 + a[i + K * l]) : 0.0);
          Rs[i + K * l] = v;
          if (i == l) rd[i] = rcp_f64(v);
        }
      __syncthreads();
      return true;
    }
  }
  // square-root-free form G = U^T D U: step j updates a_il -= a_ji a_jl / d_j (j < i <= l); the
  // owner of the next diagonal element forms its reciprocal right after its own update
  if (threadIdx.x == 0) {
    const double d0 = a[0];
    if (!(d0 > 0.0) || !isfinite(d0))
      s_bad = 1;
    else
      dinv[0] = second ? rcp_f64(d0) : rcp_f64_1(d0);
  }
  __syncthreads();
  if (s_bad) return false;
  const bool own_diag = i < K && (i % kW) == w;  // this thread holds (i, i)
  for (int j = 0; j < K; ++j) {
    if (i > j && i < K) {
      const double f = a[j + K * i] * dinv[j];
      if (own_diag && i == j + 1) {  // the next pivot first: its reciprocal overlaps the other updates
        const double v = fma(-f, a[j + K * i], a[i + K * i]);
        a[i + K * i] = v;
        if (!(v > 0.0) || !isfinite(v))
          s_bad = 1;
        else
          dinv[j + 1] = second ? rcp_f64(v) : rcp_f64_1(v);
      }
      for (int l = w; l < K; l += kW) {
        if (l < i || (l == i && i == j + 1)) continue;
        a[i + K * l] = fma(-f, a[j + K * l], a[i + K * l]);
      }
    }
    __syncthreads();
    if (s_bad) return false;
  }
  // R(i, l) = a_il / sqrt(d_i)
  if (i < K)
    for (int l = w; l < K; l += kW) {
      const double ri = rsqrt_f64(a[i + K * i]);
      Rs[i + K * l] = i <= l ? a[i + K * l] * ri : 0.0;
      if (i == l) rd[i] = ri;
    }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kS1Threads) k_site1_cholqr2(Site1Args a) {
  extern __shared__ double ys[];  // own rows, row-major with leading dimension K + 1 (odd: no bank conflicts)
  __shared__ double am[kS1MaxK * kS1MaxK];  // CTA 0: summed Gram, then the Cholesky workspace
  __shared__ double r1s[kS1MaxK * kS1MaxK];
  __shared__ double r2s[kS1MaxK * kS1MaxK];
  __shared__ double rdv[kS1MaxK];
  __shared__ double dinv[kS1MaxK];
  if (a.gate && __ldcg(a.gate) == 0) return;  // uniform: written by an earlier launch
  const int K = a.K, I1 = a.I1, tid = threadIdx.x, nthr = blockDim.x;
  const int64_t td = a.t_dev ? __ldcg(a.t_dev) : a.t;
  if (td < 1 || td > a.t) {  // outside the bound the launch was sized for: leave it to the fallback
    if (blockIdx.x == 0 && tid == 0) *a.flag = 1;
    return;
  }
  const int m = I1 * (int)td;  // rows; the grid covers the bound
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int ld = K + 1;
  // about 16 rows per CTA on the first nb CTAs (the others only take part in the barriers)
  const int nb = min((int)gridDim.x, max(1, (m + 15) / 16));
  const int rpc = (m + nb - 1) / nb;
  const int r0 = blockIdx.x * rpc;
  const int nr = (int)blockIdx.x < nb ? max(0, min(rpc, m - r0)) : 0;
  if (blockIdx.x == 0 && tid == 0) *a.flag = 0;  // read only after the next grid barrier
  // own rows of A1^T: row i + I1 r, column c <- core (i, c, r); consecutive threads, consecutive rows
  for (int x = tid; x < nr * K; x += nthr) {
    const int rr = x % nr, c = x / nr, row = r0 + rr;
    ys[rr * ld + c] = a.core0[row % I1 + I1 * (c + K * (row / I1))];
  }
  __syncthreads();
  const int npair = K * (K + 1) / 2;
  double *Gp = a.Gpart + (size_t)blockIdx.x * K * K;
  for (int pass = 0; pass < 2; ++pass) {
    // symmetric partial Gram of the own rows (CTAs without rows write nothing: only the first nb
    // partials are summed)
    for (int e = tid; e < npair && (int)blockIdx.x < nb; e += nthr) {
      int j = 0, base = 0;
      while (base + j + 1 <= e) {
        base += j + 1;
        ++j;
      }
      const int i = e - base;
      double s0 = 0.0, s1 = 0.0;
      int rr = 0;
      for (; rr + 1 < nr; rr += 2) {
        s0 = fma(ys[rr * ld + i], ys[rr * ld + j], s0);
        s1 = fma(ys[(rr + 1) * ld + i], ys[(rr + 1) * ld + j], s1);
      }
      if (rr < nr) s0 = fma(ys[rr * ld + i], ys[rr * ld + j], s0);
      Gp[i + K * j] = s0 + s1;
      Gp[j + K * i] = s0 + s1;
    }
    grid_barrier(a.bar, a.status);
    if (blockIdx.x == 0) {
      // fixed-order sum of the partials (deterministic); four loads in flight per step
      const size_t KK = (size_t)K * K;
      constexpr int kE = kS1MaxK * kS1MaxK / kS1Threads;  // elements per thread (4)
      double acc[kE];
#pragma unroll
      for (int u = 0; u < kE; ++u) acc[u] = 0.0;
      for (unsigned b0 = 0; (int)b0 < nb; b0 += 8) {
        double p[8][kE];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int u = 0; u < kE; ++u) {
            const int e = tid + u * kS1Threads;
            p[q][u] = ((int)(b0 + q) < nb && e < K * K) ? __ldcg(a.Gpart + (b0 + q) * KK + e) : 0.0;
          }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int u = 0; u < kE; ++u) acc[u] += p[q][u];
      }
#pragma unroll
      for (int u = 0; u < kE; ++u) {
        const int e = tid + u * kS1Threads;
        if (e < K * K) am[e] = acc[u];
      }
      __syncthreads();
      double *Rs = pass == 0 ? r1s : r2s;
      if (!cta_chol(am, K, Rs, rdv, pass == 1, dinv)) {
        if (tid == 0) *a.flag = 1;
      } else {
        // for the solves: S = diag(1 / R_jj) R (unit upper) to a.S, 1 / R_jj to a.rdiag
        for (int e = tid; e < K * K; e += nthr) {
          const int j = e % K;
          a.S[e] = Rs[e] * rdv[j];
        }
        if (tid < K) a.rdiag[tid] = rdv[tid];
      }
    }
    grid_barrier(a.bar, a.status);
    if (__ldcg(a.flag) != 0) return;  // every thread of every CTA reads the same value
    // Y <- Y R^{-1} row by row (warp per row, lane c owns column c): with S = diag(1/R_jj) R,
    // step j broadcasts the current y_j and lanes c > j subtract y_j S_jc; finally x_c = y_c / R_cc.
    // Two rows per warp at a time (independent chains).
    double sl[kS1MaxK];
#pragma unroll
    for (int j = 0; j < kS1MaxK; ++j) sl[j] = (lane < K && j < K) ? __ldcg(a.S + j + K * lane) : 0.0;
    const double rd = lane < K ? __ldcg(a.rdiag + lane) : 0.0;
    for (int rr = warp; rr < nr; rr += 2 * nw) {
      const int rr2 = rr + nw;
      const bool two = rr2 < nr;
      double y0 = lane < K ? ys[rr * ld + lane] : 0.0;
      double y1 = (two && lane < K) ? ys[rr2 * ld + lane] : 0.0;
#pragma unroll
      for (int j = 0; j < kS1MaxK; ++j) {
        if (j >= K) break;
        const double u0 = __shfl_sync(0xffffffffu, y0, j), u1 = __shfl_sync(0xffffffffu, y1, j);
        if (lane > j) {
          y0 = fma(-u0, sl[j], y0);
          y1 = fma(-u1, sl[j], y1);
        }
      }
      if (lane < K) {
        ys[rr * ld + lane] = y0 * rd;
        if (two) ys[rr2 * ld + lane] = y1 * rd;
      }
    }
    __syncthreads();
  }
  // Q~: column-major, or back into the core's layout (each CTA writes only the rows it read)
  for (int x = tid; x < nr * K; x += nthr) {
    const int rr = x % nr, c = x / nr, row = r0 + rr;
    if (a.core_out)
      a.core0[row % I1 + I1 * (c + K * (row / I1))] = ys[rr * ld + c];
    else
      a.Qout[row + (size_t)m * c] = ys[rr * ld + c];
  }
  if (blockIdx.x == 0)  // R~ = R2 R1 (both upper, in shared memory)
    for (int e = tid; e < K * K; e += nthr) {
      const int i = e % K, l = e / K;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int q = i;
      for (; q + 3 <= l; q += 4) {
        s0 = fma(r2s[i + K * q], r1s[q + K * l], s0);
        s1 = fma(r2s[i + K * (q + 1)], r1s[q + 1 + K * l], s1);
        s2 = fma(r2s[i + K * (q + 2)], r1s[q + 2 + K * l], s2);
        s3 = fma(r2s[i + K * (q + 3)], r1s[q + 3 + K * l], s3);
      }
      for (; q <= l; ++q) s0 = fma(r2s[i + K * q], r1s[q + K * l], s0);
      a.Rout[e] = i <= l ? (s0 + s1) + (s2 + s3) : 0.0;
    }
}

}  // namespace

// CholeskyQR2 of the site-1 matrix of core0 (1, I1, K, t) in one cooperative launch: Q~ to Qout
// (column-major (I1 t) x K) or, with core_out, back into core0 (1, I1, K, t); R~ (K x K) to Rout;
// *flag (device) = 1 when the caller must fall back to Householder (core0 is then unchanged).
// t_dev: when not null the rank is read there on the device and t is only its upper bound.
// gate: when not null, the kernel does nothing unless *gate != 0 on the device.
// Scratch: Gpart (gcap doubles), S (K x K), rdiag (K). *launched = false (nothing queued) when the
// sizes are outside the kernel's layout (K > 32, more rows than 64 CTAs hold) or gcap is too small.
int site1_cholqr2(cudaStream_t s, double *core0, int64_t I1, int64_t K, int64_t t, const int64_t *t_dev, bool core_out,
                  const int *gate, double *Gpart, int64_t gcap, double *S, double *rdiag, double *Rout, double *Qout,
                  int *flag, unsigned *bar, bool *launched) {
  *launched = false;
  const int64_t m = I1 * t;
  if (K < 1 || K > kS1MaxK || m < K || m > (int64_t)64 * kS1MaxRowsPerCta) return TNR_OK;
  int dev = 0, sms = 0;
  TNR_CK(cudaGetDevice(&dev));
  TNR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t nblk = std::min<int64_t>(std::min<int64_t>(64, sms), std::max<int64_t>(1, cdiv(m, 16)));
  const int64_t rpc = std::max<int64_t>(16, cdiv(m, nblk));  // the device's rows per CTA never exceed this
  if (rpc > kS1MaxRowsPerCta || nblk * K * K > gcap) return TNR_OK;
  const size_t smem = sizeof(double) * (size_t)(rpc * (K + 1));
  TNR_TRY(ensure_dynamic_smem((const void *)k_site1_cholqr2, smem));
  Site1Args a;
  a.core0 = core0;
  a.t_dev = t_dev;
  a.I1 = (int)I1;
  a.K = (int)K;
  a.t = (int)t;
  a.core_out = core_out ? 1 : 0;
  a.gate = gate;
  a.Gpart = Gpart;
  a.S = S;
  a.rdiag = rdiag;
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
