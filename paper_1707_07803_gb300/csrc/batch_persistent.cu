// Persistent batched TNrSVD: many independent problems solved by one kernel launch.
//
// The ordinary solve (Alg. 5.4 with Algs. 5.2 and 5.3) is a chain of short kernels with host
// round trips for the ranks the truncation chooses. For a batch of small problems that chain is
// launch- and latency-bound, so here one CTA runs the whole pipeline of one problem on its own:
// the leading-site merge (Section 6.3), the random MPO of Lemma 5.1, the 2q+2 MPO products of
// Section 5.2, after each product the exact right-to-left compression and the rounding sweeps of
// Section 5.4 (with the no-truncation certificate), the site-1 QR of Alg. 5.2, and for B the
// MPO-SVD of Alg. 5.3 with its K x K one-sided Jacobi SVD, then the outputs U, S, V. Ranks live in
// shared memory and never go back to the host until the batch is done. CTAs take problems from
// a device work queue (one atomic counter; the host orders the queue by decreasing estimated
// cost), so the launch is persistent: grid = SMs x CTAs per SM, independent of the batch size.
//
// Every dense factorisation is a one-CTA device function also used by the single-solve kernels
// (qr_tpc.cuh, svd_step.cuh, jacobi.cuh, cta_linalg.cuh). Their work areas sit in dynamic shared
// memory when they fit and otherwise in a per-problem global scratch area sized on the host from
// the structural rank bounds, so no problem that passes planning is refused on the device. The
// number of CTAs per SM (and with it the shared memory per CTA) is chosen by a small autotuner
// per shape bucket: several problems per SM share its FP64 pipes and hide each other's latency
// chains, fewer leave more of the factorisations in shared memory.
//
// Mixed precision: the products of the power iteration (the dense site-1 products, and every site
// of a zip-up product) run with FP32 operands and FP32 accumulation on the FP32 pipe (inside one
// CTA that is both cheaper and more accurate than a BF16 split: one FMA per term, about 2^-24
// relative); the roundings of the power iteration use tol_p = max(tol, kMixedTolF32), above the
// products' noise level; B = Q^T A, every QR, SVD and sweep are FP64.
//
// Rounding of a product: either the two-sweep form (the product is formed in full, then the exact
// right-to-left compression, the rounding sweeps and the site-1 step of Alg. 5.2), or the zip-up
// form (TNR_ROUND_ZIPUP: the product is rounded while it is formed, right to left, so product
// cores of rank R_k S_k never exist; the rounding sweeps and the site-1 step follow on the small
// result).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "cta_linalg.cuh"
#include "qr_tpc.cuh"

namespace tnr {
namespace {

constexpr int kBT = kStepThreads;
static_assert(kSmallThreads == kStepThreads, "the one-CTA helpers share one block size");

// One problem as the kernel sees it (device memory). Dimensions after the merge of the leading
// m sites: I, J, RA; the leading cores themselves (Ain[0..m-1]) are merged on the device.
struct BatchProblem {
  int d0, m, d, K, k, q, mixed, status;
  int zip, pad_;  // zip: products rounded as they are formed (TNR_ROUND_ZIPUP)
  uint64_t seed;
  double tol;
  int64_t max_rank;
  const double *Ain[TNR_MAX_SITES];
  int AI[TNR_MAX_SITES], AJ[TNR_MAX_SITES], AR[TNR_MAX_SITES + 1];
  int I[TNR_MAX_SITES], J[TNR_MAX_SITES], RA[TNR_MAX_SITES + 1];
  // scratch (device, per problem)
  double *merged, *merge_tmp, *omega;
  double *P0[TNR_MAX_SITES], *P1[TNR_MAX_SITES];
  int64_t pcap[TNR_MAX_SITES];
  double *tmp, *rbuf, *work, *gram, *Rm, *W, *Zr, *Sv;
  int64_t work_cap, gram_cap;  // doubles
  // zip-up scratch: carried factors (ping-pong), partial contraction, product matrix, FP32 copies
  double *zc[2], *zw, *zt;
  float *zf;
  int64_t zc_cap, zw_cap, zt_cap, zf_cap;  // elements
  // outputs (caller's buffers) and the ranks the solve chose
  double *Uc[TNR_MAX_SITES], *Vc[TNR_MAX_SITES];
  int64_t Ucap[TNR_MAX_SITES], Vcap[TNR_MAX_SITES];
  double *Sout;
  int RU[TNR_MAX_SITES + 1], RV[TNR_MAX_SITES + 1];
  double flops;  // algorithmic FP64 flops of the last solve (see addf)
};

// Shared state of the CTA working on one problem.
struct Ctx {
  double *sm;     // dynamic shared memory
  int64_t smcap;  // its size in doubles
  double *red;    // 8 * kStepWarps doubles (reductions)
  double *sc;     // 8 doubles (broadcasts)
  double *flops;  // shared accumulator of algorithmic FP64 flops (thread 0 only)
};

// Records algorithmic FP64 flops (the textbook count of each step at the ranks it ran with;
// Jacobi sweeps are not counted). All threads call it with the same value.
__device__ __forceinline__ void addf(const Ctx &c, double f) {
  if (threadIdx.x == 0) *c.flops += f;
}

// Flops of a Householder QR of an m x n matrix with p = min(m, n) reflectors plus the explicit
// m x p Q.
__device__ __forceinline__ double qr_flops(double m, double n, double p) {
  return 2 * m * n * p - (m + n) * p * p + 2 * p * p * p / 3 + 2 * m * p * p - 2 * p * p * p / 3;
}

// Row count of site k of a tall-matrix MPO made by the products: rows come from A's I (Y = A X)
// or J (Y = A^T X) and site 0 carries the K columns.
__device__ __forceinline__ int yphys(const BatchProblem &P, int rowsJ, int k) {
  return (rowsJ ? P.J[k] : P.I[k]) * (k == 0 ? P.K : 1);
}

// All threads: true when the problem has failed (uniform: no thread writes the status between
// the two barriers).
__device__ bool failed(const BatchProblem &P) {
  __syncthreads();
  const bool f = *(volatile const int *)&P.status != 0;
  __syncthreads();
  return f;
}

// Work area of `need` doubles: shared memory when it fits, else the problem's global scratch
// (sized on the host for the largest need); null (with the status set) if neither holds it.
__device__ double *pick(BatchProblem &P, const Ctx &c, int64_t need) {
  if (need <= c.smcap) return c.sm;
  if (need <= P.work_cap) return P.work;
  set_status(&P.status, TNR_ERANGE);
  return nullptr;
}

// Leading-site merge (Section 6.3): T (nr x nc x R) with core (R, I, J, R2) gives T' ((nr I) x
// (nc J) x R2), rows (a, i) -> a + nr i, columns (b, j) -> b + nc j.
__device__ const double *cta_merge(const BatchProblem &P, const Ctx &c) {
  if (P.m == 1) return P.Ain[0];
  const double *T = P.Ain[0];
  int nr = P.AI[0], nc = P.AJ[0], R = P.AR[1];
  for (int k = 1; k < P.m; ++k) {
    double *dst = ((P.m - 1 - k) % 2 == 0) ? P.merged : P.merge_tmp;
    const int I = P.AI[k], J = P.AJ[k], R2 = P.AR[k + 1];
    const int NR = nr * I, NC = nc * J, total = NR * NC * R2;
    const double *C = P.Ain[k];
    for (int idx = threadIdx.x; idx < total; idx += kBT) {
      const int row = idx % NR, col = (idx / NR) % NC, s = idx / (NR * NC);
      const int a = row % nr, i = row / nr, b = col % nc, j = col / nc;
      double acc = 0.0;
      for (int r = 0; r < R; ++r) acc = fma(T[a + nr * (b + nc * r)], C[r + R * (i + I * (j + J * s))], acc);
      dst[idx] = acc;
    }
    __syncthreads();
    addf(c, 2.0 * total * R);
    T = dst;
    nr = NR;
    nc = NC;
    R = R2;
  }
  return T;
}

// Dense site-1 product with FP32 operands and FP32 accumulation: every operand is rounded to FP32
// once (staged in the work area; on GB300 a double->float conversion issues on the FP64 pipe, so it
// is done once per element, not once per multiply-add), then one FMA per term on the FP32 pipe.
// A (1, I, J, R2), X (1, Ny, Kx, S2), Y (Xo, Kx, R2 S2).
__device__ void cta_product_f32(BatchProblem &P, const Ctx &c, const double *A, int I, int J, int R2,
                                const double *X, int Kx, int S2, int trans, double *Y) {
  const int Xo = trans ? J : I, Ny = trans ? I : J;
  const int na = I * J * R2, nx = Ny * Kx * S2;
  double *area = pick(P, c, ((int64_t)na + nx + 1) / 2);
  if (!area) return;
  float *af = reinterpret_cast<float *>(area), *xf = af + na;
  for (int e = threadIdx.x; e < na + nx; e += kBT) {
    if (e < na)
      af[e] = (float)A[e];
    else
      xf[e - na] = (float)X[e - na];
  }
  __syncthreads();
  const int total = Xo * Kx * R2 * S2;
  for (int idx = threadIdx.x; idx < total; idx += kBT) {
    const int xo = idx % Xo, t = idx / Xo, cc = t % Kx, rs2 = t / Kx;
    const int r2 = rs2 % R2, s2 = rs2 / R2;
    const int a0 = trans ? I * (xo + J * r2) : xo + I * J * r2;
    const int as = trans ? 1 : I;
    const int x0 = Ny * (cc + Kx * s2);
    float acc = 0.f;
    for (int y = 0; y < Ny; ++y) acc = fmaf(af[a0 + as * y], xf[x0 + y], acc);
    Y[idx] = (double)acc;
  }
  __syncthreads();
}

// Y = op(A) X for every site (Section 5.2); output core (R S, Xo, Kx, R2 S2), bonds r + R s.
// X: cores Xc with ranks XR, rows Ny = (trans ? I : J), K columns on site 0.
__device__ void cta_contract(BatchProblem &P, const Ctx &c, const double *A0, int trans, const double *const *Xc,
                             const int *XR, double *const *Yc, int *YR, bool mixed) {
  for (int k = 0; k < P.d; ++k) {
    const int R = P.RA[k], I = P.I[k], J = P.J[k], R2 = P.RA[k + 1];
    const int S = XR[k], S2 = XR[k + 1];
    const int Kx = k == 0 ? P.K : 1;
    const int Xo = trans ? J : I, Ny = trans ? I : J;
    const int64_t total = (int64_t)R * S * Xo * Kx * R2 * S2;
    if (total > P.pcap[k]) {
      set_status(&P.status, TNR_ENOMEM);
      return;
    }
    const double *A = k == 0 ? A0 : P.Ain[P.m - 1 + k];
    const double *X = Xc[k];
    double *Y = Yc[k];
    if (mixed && R == 1 && S == 1 && Ny >= 16) {
      cta_product_f32(P, c, A, I, J, R2, X, Kx, S2, trans, Y);
      continue;
    }
    const int RS = R * S, nt = (int)total;
    const int as = trans ? R : R * I;
    for (int idx = threadIdx.x; idx < nt; idx += kBT) {
      int t = idx;
      const int rs = t % RS;
      t /= RS;
      const int xo = t % Xo;
      t /= Xo;
      const int cc = t % Kx;
      const int rs2 = t / Kx;
      const int r = rs % R, s = rs / R, r2 = rs2 % R2, s2 = rs2 / R2;
      const double *xp = X + s + S * (Ny * (cc + Kx * s2));
      const double *ap = trans ? A + r + R * (I * (xo + J * r2)) : A + r + R * (xo + I * (J * r2));
      double acc = 0.0;
      for (int y = 0; y < Ny; ++y) acc = fma(ap[as * y], xp[S * y], acc);
      Y[idx] = acc;
    }
    addf(c, 2.0 * (double)total * Ny);
  }
  if (threadIdx.x == 0) {
    YR[0] = 1;
    for (int k = 0; k < P.d; ++k) YR[k + 1] = P.RA[k + 1] * XR[k + 1];
  }
  __syncthreads();
}

// Y = op(A) X rounded while it is formed (zip-up, TNR_ROUND_ZIPUP), right to left. With C the
// factor carried from site k+1 ((R_{k+1} S_{k+1}) x t, bond r + R s), site k forms
//   T[(r + R s), x, c, b] = sum_y sum_{r2} A_k(r, x, y, r2) sum_{s2} X_k(s, y, c, s2) C[(r2 + R2 s2), b]
// one value of the shared physical index y at a time (W = X_k(:, y, :, :) C is S Kx R2 t values),
// so neither the product core nor a full partial contraction is stored. For k >= 1, T is the
// (R S) x (Xo Kx t) matrix of the truncated-SVD step (svd_step_cta): the smallest rank r >= 1 with
// discarded squared singular values <= tol_z^2 ||T||_F^2 / (d - 1), then r <= max_rank; core k
// becomes the r kept right singular vectors (orthonormal rows) and U diag(s) the next C. Site 0
// absorbs the last C. mixed: X_k, C and A_k are rounded to FP32 once per site and the sums run in
// FP32; T and the SVD stay FP64. Output ranks go to YR.
__device__ __noinline__ void cta_zipup(BatchProblem &P, const Ctx &c, const double *A0, int trans, const double *const *Xc,
                          const int *XR, double *const *Yc, int *YR, double tol_z, int64_t max_rank, bool mixed) {
  __shared__ int s_t;
  const int d = P.d;
  double *C = P.zc[0], *Cn = P.zc[1];
  if (threadIdx.x == 0) {
    C[0] = 1.0;
    s_t = 1;
    YR[0] = 1;
    YR[d] = 1;
  }
  __syncthreads();
  for (int k = d - 1; k >= 0; --k) {
    const int t = s_t;
    const int R = P.RA[k], I = P.I[k], J = P.J[k], R2 = P.RA[k + 1];
    const int S = XR[k], S2 = XR[k + 1];
    const int Kx = k == 0 ? P.K : 1;
    const int Xo = trans ? J : I, Ny = trans ? I : J;
    const int RS = R * S, w = Xo * Kx * t;
    const double *A = k == 0 ? A0 : P.Ain[P.m - 1 + k];
    const double *X = Xc[k];
    const int64_t nT = (int64_t)RS * w, nW = (int64_t)S * Kx * R2 * t;
    double *T = k == 0 ? Yc[0] : P.zt;
    if ((k == 0 && nT > P.pcap[0]) || (k > 0 && nT > P.zt_cap) || nW > P.zw_cap) {
      set_status(&P.status, k == 0 ? TNR_ENOMEM : TNR_ERANGE);
      return;
    }
    for (int64_t i = threadIdx.x; i < nT; i += kBT) T[i] = 0.0;
    // A_k(r, x, y, r2) at a_base(r, x, r2) + a_y * y
    const int a_y = trans ? R : R * I;
    const int nA = R * I * J * R2, nX = S * Ny * Kx * S2, nC = R2 * S2 * t;
    float *Af = P.zf, *Xf = Af + nA, *Cf = Xf + nX, *Wf = Cf + nC;
    if (mixed) {
      if ((int64_t)nA + nX + nC + nW > P.zf_cap) {
        set_status(&P.status, TNR_ERANGE);
        return;
      }
      for (int e = threadIdx.x; e < nA + nX + nC; e += kBT) {
        if (e < nA)
          Af[e] = (float)A[e];
        else if (e < nA + nX)
          Xf[e - nA] = (float)X[e - nA];
        else
          Cf[e - nA - nX] = (float)C[e - nA - nX];
      }
    }
    __syncthreads();
    for (int y = 0; y < Ny; ++y) {
      // W[s + S (cc + Kx (r2 + R2 b))] = sum_{s2} X_k(s, y, cc, s2) C[(r2 + R2 s2) + R2 S2 b]
      for (int idx = threadIdx.x; idx < (int)nW; idx += kBT) {
        const int s_ = idx % S, u = idx / S, cc = u % Kx, v = u / Kx, r2 = v % R2, b = v / R2;
        const int x0 = s_ + S * (y + Ny * cc), xs = S * Ny * Kx;
        const int c0 = r2 + R2 * S2 * b, cs = R2;
        if (mixed) {
          float acc = 0.f, acc1 = 0.f;
          int s2 = 0;
          for (; s2 + 1 < S2; s2 += 2) {  // two terms in flight
            acc = fmaf(Xf[x0 + xs * s2], Cf[c0 + cs * s2], acc);
            acc1 = fmaf(Xf[x0 + xs * (s2 + 1)], Cf[c0 + cs * (s2 + 1)], acc1);
          }
          if (s2 < S2) acc = fmaf(Xf[x0 + xs * s2], Cf[c0 + cs * s2], acc);
          Wf[idx] = acc + acc1;
        } else {
          double acc = 0.0, acc1 = 0.0;
          int s2 = 0;
          for (; s2 + 1 < S2; s2 += 2) {
            acc = fma(X[x0 + xs * s2], C[c0 + cs * s2], acc);
            acc1 = fma(X[x0 + xs * (s2 + 1)], C[c0 + cs * (s2 + 1)], acc1);
          }
          if (s2 < S2) acc = fma(X[x0 + xs * s2], C[c0 + cs * s2], acc);
          P.zw[idx] = acc + acc1;
        }
      }
      __syncthreads();
      // T[(r + R s) + RS (x + Xo (cc + Kx b))] += sum_{r2} A_k(r, x, y, r2) W[s, cc, r2, b]
      for (int idx = threadIdx.x; idx < (int)nT; idx += kBT) {
        const int rs = idx % RS, u = idx / RS, x = u % Xo, v = u / Xo, cc = v % Kx, b = v / Kx;
        const int r = rs % R, s_ = rs / R;
        const int a0 = (trans ? r + R * (I * x) : r + R * x) + a_y * y, as = R * I * J;
        const int w0 = s_ + S * (cc + Kx * R2 * b), ws = S * Kx;
        if (mixed) {
          float acc = 0.f, acc1 = 0.f;
          int r2 = 0;
          for (; r2 + 1 < R2; r2 += 2) {  // two terms in flight
            acc = fmaf(Af[a0 + as * r2], Wf[w0 + ws * r2], acc);
            acc1 = fmaf(Af[a0 + as * (r2 + 1)], Wf[w0 + ws * (r2 + 1)], acc1);
          }
          if (r2 < R2) acc = fmaf(Af[a0 + as * r2], Wf[w0 + ws * r2], acc);
          T[idx] += (double)(acc + acc1);
        } else {
          double acc = 0.0, acc1 = 0.0;
          int r2 = 0;
          for (; r2 + 1 < R2; r2 += 2) {
            acc = fma(A[a0 + as * r2], P.zw[w0 + ws * r2], acc);
            acc1 = fma(A[a0 + as * (r2 + 1)], P.zw[w0 + ws * (r2 + 1)], acc1);
          }
          if (r2 < R2) acc = fma(A[a0 + as * r2], P.zw[w0 + ws * r2], acc);
          T[idx] += acc + acc1;
        }
      }
      __syncthreads();
    }
    if (!mixed) addf(c, 2.0 * Ny * ((double)nW * S2 + (double)nT * R2));  // FP64 work only
    if (k == 0) break;
    // truncated SVD of T ((R S) x w), threshold relative to ||T||_F
    double nrm2;
    {
      double a = 0.0;
      for (int64_t i = threadIdx.x; i < nT; i += kBT) a = fma(T[i], T[i], a);
      nrm2 = cta_sum(a, kBT, c.red, c.sc);
    }
    if (svd_step_work(RS, w) > P.work_cap || (RS < w ? RS : w) > kStepMaxN) {
      set_status(&P.status, TNR_ERANGE);
      return;
    }
    const double delta2 = tol_z * tol_z * nrm2 / (double)(d - 1);
    double *work = pick(P, c, svd_step_work(RS, w));
    if (!work) return;
    const int r = svd_step_cta(T, RS, w, delta2, max_rank, Yc[k], Cn, work, &P.status);
    {
      const double mm = RS > w ? RS : w, n = RS > w ? w : RS;
      addf(c, 2 * mm * n * n - 2 * n * n * n / 3);
    }
    if (threadIdx.x == 0) {
      YR[k] = r;
      s_t = r;
    }
    double *tmpc = C;
    C = Cn;
    Cn = tmpc;
    __syncthreads();
  }
}

// Exact right-to-left compression (as the single solve's compression sweep): for k = d-1..1,
// M_k (t x w) = L Q_k by the column-pivoted QR of M_k^T that stops at the cutoff; Q_k becomes
// core k, L is absorbed into core k-1. Bonds whose w exceeds the one-CTA QR (64) keep their
// core. Returns true when every bond was compressed (cores 1..d-1 right-orthonormal).
__device__ bool cta_compress(BatchProblem &P, const Ctx &c, double *const *core, int *R, int rowsJ, double cut) {
  __shared__ int64_t s_r;
  bool all = true;
  for (int k = P.d - 1; k >= 1; --k) {
    const int t = R[k], w = yphys(P, rowsJ, k) * R[k + 1];
    const int64_t need = (qr_tpc_bytes(w, t) + 7) / 8;
    if (w > 64 || need > (c.smcap > P.work_cap ? c.smcap : P.work_cap)) {
      all = false;
      continue;
    }
    double *area = pick(P, c, need);
    QrSmallArgs q;
    q.src = core[k];
    q.lds = t;
    q.m = w;
    q.n = t;
    q.trans_src = 1;
    q.pivot = 1;
    q.trans_q = 1;
    q.trans_r = 1;
    q.cut_rel = cut;
    q.Q = core[k];
    q.ldq = 0;
    q.R = P.rbuf;
    q.ldr = t;
    q.r_out = &s_r;
    qr_tpc_cta(q, area);
    __syncthreads();
    const int r = (int)s_r;
    {
      const double M = w, N = t, rr = r, rows = (double)R[k - 1] * yphys(P, rowsJ, k - 1);
      addf(c, 4 * M * N * rr - 2 * (M + N) * rr * rr + 4 * rr * rr * rr / 3 + 2 * M * rr * rr - 2 * rr * rr * rr / 3 +
                  2 * rows * N * rr);
    }
    cta_absorb_right(core[k - 1], R[k - 1] * yphys(P, rowsJ, k - 1), t, P.rbuf, r, c.sm, (int)c.smcap);
    if (threadIdx.x == 0) R[k] = r;
    __syncthreads();
  }
  return all;
}

// No-truncation certificate (the Gram recurrence of the fused rounding kernel) on cores in
// global memory; valid when cores 1..d-1 are right-orthonormal. True (uniform) when no bond
// would be truncated by the rounding.
__device__ bool cta_certified(BatchProblem &P, const Ctx &c, double *const *core, const int *R, int rowsJ,
                              double tol, int64_t max_rank) {
  __shared__ int goff[TNR_MAX_SITES];
  __shared__ int s_ok;
  const int d = P.d;
  if (threadIdx.x == 0) {
    int off = 0, ok = 1;
    for (int k = 1; k < d; ++k) {
      goff[k] = off;
      off += R[k] * R[k];
      if (R[k] > 32 || (max_rank > 0 && R[k] > max_rank)) ok = 0;
    }
    if (off > P.gram_cap) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) {
    __syncthreads();
    return false;
  }
  double *gram = P.gram;
  cta_tn_sym(gram + goff[1], core[0], core[0], R[0] * yphys(P, rowsJ, 0), R[1]);
  addf(c, (double)R[0] * yphys(P, rowsJ, 0) * R[1] * (R[1] + 1));
  for (int k = 1; k + 1 < d; ++k) {
    const int r = R[k], w = yphys(P, rowsJ, k) * R[k + 1];
    addf(c, 2.0 * r * r * w + (double)r * yphys(P, rowsJ, k) * R[k + 1] * (R[k + 1] + 1));
    cta_gemm(P.tmp, gram + goff[k], r, core[k], r, r, w, r);  // T = G_k C_k (r x phys r')
    cta_tn_sym(gram + goff[k + 1], core[k], P.tmp, r * yphys(P, rowsJ, k), R[k + 1]);
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < R[1]; ++b) t += gram[goff[1] + b + R[1] * b];
    c.sc[0] = tol * tol * t / (double)(d - 1);  // delta^2
  }
  __syncthreads();
  const double delta2 = c.sc[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 1 + warp; k < d; k += kStepWarps) {
    const double lb = warp_lambda_min_bound(gram + goff[k], R[k]);
    if (lane == 0 && !(lb > delta2 * (1.0 + 1e-6))) atomicExch(&s_ok, 0);
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

// Rounding (Section 5.4): left-to-right Householder QR sweep, then the right-to-left truncated
// SVD sweep (the loop of Alg. 5.2); skipped when the certificate shows nothing would be cut.
__device__ void cta_round(BatchProblem &P, const Ctx &c, double *const *core, int *R, int rowsJ, double tol,
                          int64_t max_rank, bool certify) {
  const int d = P.d;
  if (d < 2) return;
  if (certify && cta_certified(P, c, core, R, rowsJ, tol, max_rank)) return;
  for (int k = 0; k + 1 < d; ++k) {
    const int rows = R[k] * yphys(P, rowsJ, k), cols = R[k + 1];
    const int nq = rows < cols ? rows : cols;
    double *A = pick(P, c, (int64_t)rows * cols + nq);
    if (!A) return;
    for (int i = threadIdx.x; i < rows * cols; i += kBT) A[i] = core[k][i];
    __syncthreads();
    cta_qr(A, rows, cols, P.rbuf, A + rows * cols, c.red, c.sc);
    for (int i = threadIdx.x; i < rows * nq; i += kBT) core[k][i] = A[i];
    const int w = yphys(P, rowsJ, k + 1) * R[k + 2];
    addf(c, qr_flops(rows, cols, nq) + 2.0 * nq * cols * w);
    cta_gemm(P.tmp, P.rbuf, nq, core[k + 1], cols, nq, w, cols);  // R (nq x cols) C_{k+1}
    for (int i = threadIdx.x; i < nq * w; i += kBT) core[k + 1][i] = P.tmp[i];
    if (threadIdx.x == 0) R[k + 1] = nq;
    __syncthreads();
  }
  // ||Y||_F^2 = ||last core||_F^2 (the other cores are left-orthonormal now)
  double nrm2;
  {
    const int n = R[d - 1] * yphys(P, rowsJ, d - 1) * R[d];
    const double *x = core[d - 1];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kBT) s = fma(x[i], x[i], s);
    nrm2 = cta_sum(s, n, c.red, c.sc);
  }
  const double delta2 = tol * tol * nrm2 / (double)(d - 1);
  for (int k = d - 1; k >= 1; --k) {
    const int t = R[k], w = yphys(P, rowsJ, k) * R[k + 1];
    double *work = pick(P, c, svd_step_work(t, w));
    if (!work) return;
    const int r = svd_step_cta(core[k], t, w, delta2, max_rank, core[k], P.rbuf, work, &P.status);
    {
      const double mm = t > w ? t : w, n = t > w ? w : t;
      addf(c, 2 * mm * n * n - 2 * n * n * n / 3 + 2.0 * R[k - 1] * yphys(P, rowsJ, k - 1) * t * r);
    }
    cta_absorb_right(core[k - 1], R[k - 1] * yphys(P, rowsJ, k - 1), t, P.rbuf, r, c.sm, (int)c.smcap);
    if (threadIdx.x == 0) R[k] = r;
    __syncthreads();
  }
}

// Site-1 matrix of Algs. 5.2/5.3: core (1, I1, K, t) -> A1^T ((I1 t) x K) in A (ld m), then its
// Householder QR: A <- Q~ (explicit), Rm <- R~ (K x K).
__device__ double *cta_site1_qr(BatchProblem &P, const Ctx &c, const double *core0, int I1, int t, int64_t extra) {
  const int K = P.K, m = I1 * t;
  if (m < K) {
    set_status(&P.status, TNR_EINVAL);
    return nullptr;
  }
  const int64_t need = (int64_t)m * K + K;
  double *A = pick(P, c, need + extra);
  if (!A) return nullptr;
  for (int idx = threadIdx.x; idx < m * K; idx += kBT) {
    const int i = idx % I1, cc = (idx / I1) % K, r = idx / (I1 * K);
    A[(i + I1 * r) + m * cc] = core0[idx];
  }
  __syncthreads();
  cta_qr(A, m, K, P.Rm, A + (int64_t)m * K, c.red, c.sc);
  addf(c, qr_flops(m, K, K));
  return A;
}

// MPO-QR with integrated rounding (Alg. 5.2 + Section 5.4) of a tall-matrix MPO. zipped: the
// MPO comes from a zip-up product (cores 1..d-1 right-orthonormal already, no compression). The
// Gram no-truncation certificate is not used then: the zip-up truncates in a non-orthonormal gauge
// and can keep directions whose canonical Schmidt values lie far below sqrt(eps) ||Y||, which a
// Gram matrix formed in FP64 cannot resolve; the sweeps (QR and SVD of the cores) do resolve them.
__device__ void cta_orthogonalize(BatchProblem &P, const Ctx &c, double *const *core, int *R, int rowsJ, double tol,
                                  int64_t max_rank, bool mixed_product, bool zipped) {
  bool right_orth = false;
  if (!zipped && tol > 0.0) right_orth = cta_compress(P, c, core, R, rowsJ, compress_cut(tol, mixed_product));
  cta_round(P, c, core, R, rowsJ, tol, max_rank, right_orth);
  if (failed(P)) return;
  const int I1 = rowsJ ? P.J[0] : P.I[0], K = P.K, t = R[1], m = I1 * t;
  double *A = cta_site1_qr(P, c, core[0], I1, t, 0);
  if (!A) return;
  for (int idx = threadIdx.x; idx < m * K; idx += kBT) {
    const int i = idx % I1, cc = (idx / I1) % K, r = idx / (I1 * K);
    core[0][idx] = A[(i + I1 * r) + m * cc];
  }
  __syncthreads();
}

// MPO-SVD (Alg. 5.3 + Section 5.4) of B = Z^T (Z = A^T Q, cores P1 / ranks R): rounding, site-1
// QR M^T = Q~ R~, one-sided Jacobi R~^T = W S Zr^T, V^(1) from Q~ Zr (first k columns).
__device__ void cta_mpo_svd(BatchProblem &P, const Ctx &c, double *const *core, int *R, bool zipped) {
  bool right_orth = false;  // zipped: no compression and no certificate (see cta_orthogonalize)
  if (!zipped && P.tol > 0.0) right_orth = cta_compress(P, c, core, R, 1, compress_cut(P.tol, false));
  cta_round(P, c, core, R, 1, P.tol, P.max_rank, right_orth);
  if (failed(P)) return;
  const int J1 = P.J[0], K = P.K, t = R[1], m = J1 * t, kout = P.k;
  const int64_t qneed = (int64_t)m * K + K, jneed = 2 * (int64_t)K * K + 2 * K + jacobi_mixed_work(K);
  // Jacobi area after the QR's when both fit shared memory, else on its own
  const bool both_sm = qneed + jneed <= c.smcap;
  double *A = cta_site1_qr(P, c, core[0], J1, t, both_sm ? 0 : jneed);
  if (!A) return;
  double *G = both_sm ? c.sm + qneed : (jneed <= c.smcap && A != c.sm ? c.sm : A + qneed);
  double *Vj = G + K * K, *nrm = Vj + K * K, *inv = nrm + K;
  for (int idx = threadIdx.x; idx < K * K; idx += kBT) {
    const int i = idx % K, j = idx / K;
    G[idx] = P.Rm[j + K * i];  // R~^T
    Vj[idx] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps_mixed(G, Vj, K, nrm, inv + K);
  for (int j = threadIdx.x; j < K; j += kBT) {
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < K; i += 2) {
      s0 = fma(G[i + K * j], G[i + K * j], s0);
      s1 = fma(G[i + 1 + K * j], G[i + 1 + K * j], s1);
    }
    if (i < K) s0 = fma(G[i + K * j], G[i + K * j], s0);
    const double sj = sqrt(s0 + s1);
    if (!isfinite(sj)) set_status(&P.status, TNR_ENONFINITE);
    nrm[j] = sj;
    inv[j] = sj > 0.0 ? 1.0 / sj : 0.0;
  }
  __syncthreads();
  // order by descending singular value (stable): W[:, rank] = G[:, j] / s_j, Zr[:, rank] = V[:, j]
  for (int j = threadIdx.x; j < K; j += kBT) {
    const double sj = nrm[j];
    int rank = 0;
    for (int i = 0; i < K; ++i) rank += (nrm[i] > sj || (nrm[i] == sj && i < j)) ? 1 : 0;
    const double iv = inv[j];
    for (int i = 0; i < K; ++i) {
      P.W[i + K * rank] = G[i + K * j] * iv;
      P.Zr[i + K * rank] = Vj[i + K * j];
    }
    P.Sv[rank] = sj;
  }
  __syncthreads();
  cta_gemm(P.tmp, A, m, P.Zr, K, m, K, K);  // V = Q~ Zr (m x K)
  addf(c, 2.0 * m * K * K);
  if ((int64_t)J1 * kout * t > P.Vcap[0]) {
    set_status(&P.status, TNR_ENOMEM);
    return;
  }
  for (int idx = threadIdx.x; idx < J1 * kout * t; idx += kBT) {
    const int i = idx % J1, cc = (idx / J1) % kout, r = idx / (J1 * kout);
    P.Vc[0][idx] = P.tmp[(i + J1 * r) + m * cc];
  }
  __syncthreads();
}

// The whole solve of one problem by the calling CTA.
__device__ void cta_solve(BatchProblem &P, const Ctx &c) {
  __shared__ int RY0[TNR_MAX_SITES + 1], RY1[TNR_MAX_SITES + 1], RO[TNR_MAX_SITES + 1];
  const int d = P.d, K = P.K;
  if (threadIdx.x == 0) {
    *c.flops = 0.0;
    P.status = 0;  // each launch solves the problem afresh
  }
  __syncthreads();
  const double *A0 = cta_merge(P, c);
  // Lemma 5.1: Omega^(1) (J1 x K) then the vectors of sites 2..d, in draw order
  int64_t omega_len = (int64_t)P.J[0] * K;
  for (int k = 1; k < d; ++k) omega_len += P.J[k];
  for (int64_t m = threadIdx.x; m < omega_len; m += kBT) P.omega[m] = omega_normal(P.seed, (uint64_t)m);
  __shared__ const double *Oc[TNR_MAX_SITES];
  if (threadIdx.x == 0) {
    int64_t pos = 0;
    for (int k = 0; k < d; ++k) {
      Oc[k] = P.omega + pos;
      pos += k == 0 ? (int64_t)P.J[0] * K : P.J[k];
      RO[k] = 1;
    }
    RO[d] = 1;
  }
  __syncthreads();
  const bool mixed = P.mixed != 0, zip = P.zip != 0;
  const double tol_p = mixed ? fmax(P.tol, kMixedTolF32) : P.tol;
  // Y = op(A) X followed by MPO-QR: formed in full and compressed, or rounded as it is formed
  auto product_qr = [&](int trans, const double *const *Xc, const int *XR, double *const *Yc, int *YR) {
    if (zip)
      cta_zipup(P, c, A0, trans, Xc, XR, Yc, YR, tol_p, P.max_rank, mixed);
    else
      cta_contract(P, c, A0, trans, Xc, XR, Yc, YR, mixed);
    if (failed(P)) return;
    cta_orthogonalize(P, c, Yc, YR, trans, tol_p, P.max_rank, mixed, zip);
  };
  product_qr(0, Oc, RO, P.P0, RY0);  // Y = A Omega
  if (failed(P)) return;
  for (int it = 0; it < P.q; ++it) {
    product_qr(1, P.P0, RY0, P.P1, RY1);  // A^T Q
    if (failed(P)) return;
    product_qr(0, P.P1, RY1, P.P0, RY0);  // A Q
    if (failed(P)) return;
  }
  if (zip)  // Z = A^T Q = B^T (FP64)
    cta_zipup(P, c, A0, 1, P.P0, RY0, P.P1, RY1, P.tol, P.max_rank, false);
  else
    cta_contract(P, c, A0, 1, P.P0, RY0, P.P1, RY1, false);
  if (failed(P)) return;
  cta_mpo_svd(P, c, P.P1, RY1, zip);
  if (failed(P)) return;
  // U^(1) = Q^(1) x_3 W[:, :k] (Section 5.4); cores 2..d of U and V are those of Q and Z
  const int I1 = P.I[0], t = RY0[1], kout = P.k;
  if ((int64_t)I1 * kout * t > P.Ucap[0]) {
    set_status(&P.status, TNR_ENOMEM);
    return;
  }
  const double *Q0 = P.P0[0];
  addf(c, 2.0 * I1 * kout * t * K);
  for (int idx = threadIdx.x; idx < I1 * kout * t; idx += kBT) {
    const int i = idx % I1, cc = (idx / I1) % kout, r = idx / (I1 * kout);
    const double *q = Q0 + i + I1 * K * r;
    const double *w = P.W + K * cc;
    double acc = 0.0;
    for (int l = 0; l < K; ++l) acc = fma(q[I1 * l], w[l], acc);
    P.Uc[0][idx] = acc;
  }
  for (int k = 1; k < d; ++k) {
    const int ue = RY0[k] * P.I[k] * RY0[k + 1], ve = RY1[k] * P.J[k] * RY1[k + 1];
    if (ue > P.Ucap[k] || ve > P.Vcap[k]) {
      set_status(&P.status, TNR_ENOMEM);
      return;
    }
    for (int i = threadIdx.x; i < ue; i += kBT) P.Uc[k][i] = P.P0[k][i];
    for (int i = threadIdx.x; i < ve; i += kBT) P.Vc[k][i] = P.P1[k][i];
  }
  for (int i = threadIdx.x; i < kout; i += kBT) P.Sout[i] = P.Sv[i];
  for (int k = threadIdx.x; k <= d; k += kBT) {
    P.RU[k] = RY0[k];
    P.RV[k] = RY1[k];
  }
  if (threadIdx.x == 0) P.flops = *c.flops;
  __syncthreads();
}

// Persistent kernel: each CTA takes problems from the queue until it is empty.
__global__ void __launch_bounds__(kBT, 2) k_batch_solve(BatchProblem *probs, int n, int *queue, int64_t smcap) {
  extern __shared__ double sm[];
  __shared__ double red[8 * kStepWarps];
  __shared__ double sc[8];
  __shared__ int s_p;
  __shared__ double s_flops;
  Ctx c;
  c.sm = sm;
  c.smcap = smcap;
  c.red = red;
  c.sc = sc;
  c.flops = &s_flops;
  for (;;) {
    if (threadIdx.x == 0) s_p = atomicAdd(queue, 1);
    __syncthreads();
    const int p = s_p;
    __syncthreads();
    if (p >= n) break;
    cta_solve(probs[p], c);
  }
}

// ---------------------------------------------------------------------------------------
// Host side: planning, workspace, launch configuration, autotuning, graph capture.
// ---------------------------------------------------------------------------------------

constexpr int64_t kIntMax = 2147483647;

int64_t pow2_ceil(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Plans problem `pr`, carves its scratch from `ar` and (when bp is not null) fills its
// descriptor. cost: an estimate of its FP64 work, for the queue order.
int plan_problem(const tnr_problem &pr, Arena &ar, BatchProblem *bp, double *cost, int64_t *bucket) {
  if (!pr.A || !pr.U || !pr.V || !pr.S || pr.k < 1 || pr.p < 0 || pr.q < 0) return TNR_EINVAL;
  if (pr.A->dtype != TNR_F64) return TNR_EINVAL;  // the kernel reads float64 cores
  if (pr.opts.precision != TNR_FP64 && pr.opts.precision != TNR_MIXED) return TNR_EINVAL;
  if (pr.opts.rounding != TNR_ROUND_TWO_SWEEP && pr.opts.rounding != TNR_ROUND_ZIPUP) return TNR_EINVAL;
  const bool zip = pr.opts.rounding == TNR_ROUND_ZIPUP;
  const bool mixed = pr.opts.precision == TNR_MIXED;
  const int64_t K = (int64_t)pr.k + pr.p;
  Plan P;
  TNR_TRY(make_plan(pr.A, K, &pr.opts, P));
  // Zip-up: no product core is formed. Bond k of a rounded product holds at most
  // zq[k] = min(R_k sq_k, X_k zq[k+1], max_rank) (rows of T_k, columns of T_k, the cap), and
  // every core the solve keeps (Y, Q, Z, V) fits zq[k] X_k K_k zq[k+1].
  int64_t zq[TNR_MAX_SITES + 1];
  int64_t zc_cap = 1, zw_cap = 1, zt_cap = 1, zf_cap = 1, zsvd = 1;
  if (zip) {
    zq[0] = 1;
    zq[P.d] = 1;
    for (int k = P.d - 1; k >= 1; --k) {
      const int64_t X = std::max(P.I[k], P.J[k]);
      int64_t v = std::min(P.RA[k] * P.sq[k], X * zq[k + 1]);
      if (pr.opts.max_rank > 0) v = std::min<int64_t>(v, pr.opts.max_rank);
      zq[k] = std::max<int64_t>(v, 1);
    }
    for (int k = 0; k < P.d; ++k) {
      const int64_t X = std::max(P.I[k], P.J[k]), Kx = k == 0 ? K : 1;
      const int64_t S = k == 0 ? 1 : P.sq[k], S2 = P.sq[k + 1], R = P.RA[k], R2 = P.RA[k + 1];
      const int64_t t = zq[k + 1], rows = R * S, w = X * Kx * t;
      P.pcap[k] = zq[k] * X * Kx * zq[k + 1];
      zw_cap = std::max(zw_cap, S * Kx * R2 * t);
      if (k >= 1) {
        zt_cap = std::max(zt_cap, rows * w);
        zc_cap = std::max(zc_cap, rows * zq[k]);
        if (std::min(rows, w) > kStepMaxN) return TNR_ENOMEM;  // one-CTA SVD step limit
        zsvd = std::max(zsvd, svd_step_work(rows, w));
      }
      if (mixed) zf_cap = std::max(zf_cap, R * P.I[k] * P.J[k] * R2 + S * X * Kx * S2 + R2 * S2 * t + S * Kx * R2 * t);
    }
    // the rounding sweeps, site-1 steps and outputs then run on bonds of at most zq
    P.L.maxcore = 1;
    P.L.maxbond = 1;
    for (int k = 0; k < P.d; ++k) {
      P.L.maxcore = std::max(P.L.maxcore, P.pcap[k]);
      P.L.maxbond = std::max(P.L.maxbond, std::max(zq[k], zq[k + 1]));
    }
    P.L.maxcore = std::max(P.L.maxcore, std::max(P.I[0], P.J[0]) * K * zq[1]);
    for (int k = 0; k <= P.d; ++k) P.sq[k] = std::min(P.sq[k], zq[k]);  // bonds of every rounded MPO
  }
  if (pr.U->d != P.d || pr.V->d != P.d) return TNR_EINVAL;
  const tnr_mpo &A = *pr.A;
  // every index the kernel forms is a 32-bit int
  int64_t maxA = 1;
  for (int k = 0; k < A.d; ++k) maxA = std::max(maxA, A.R[k] * A.I[k] * A.J[k] * A.R[k + 1]);
  if (maxA > kIntMax || P.merged_elems > kIntMax || P.omega_len > kIntMax) return TNR_ERANGE;
  for (int k = 0; k < P.d; ++k)
    if (P.pcap[k] > kIntMax) return TNR_ERANGE;
  // work area bound (doubles): every factorisation's need at the structural bounds
  int64_t wc = zip ? zsvd : 1;
  for (int k = 0; k < P.d; ++k) {
    const int64_t X = std::max(P.I[k], P.J[k]), Kx = k == 0 ? K : 1;
    const int64_t t = zip ? zq[k] : P.RA[k] * P.sq[k], t2 = zip ? zq[k + 1] : P.RA[k + 1] * P.sq[k + 1];
    if (k + 1 < P.d) {
      const int64_t rows = t * X * Kx;
      wc = std::max(wc, rows * t2 + std::min(rows, t2));  // L->R QR
    }
    if (k >= 1) {
      const int64_t w = X * t2;
      wc = std::max(wc, svd_step_work(t, w));                               // R->L SVD step
      wc = std::max(wc, (qr_tpc_bytes(std::min<int64_t>(64, w), t) + 7) / 8);  // compression
    }
  }
  {
    const int64_t X0 = std::max(P.I[0], P.J[0]), t1 = zip ? zq[1] : P.RA[1] * P.sq[1];
    wc = std::max(wc, X0 * t1 * K + K + 2 * K * K + 2 * K + jacobi_mixed_work(K));  // site-1 QR, K x K SVD
    wc = std::max(wc, (P.I[0] * P.J[0] * P.RA[1] + X0 * K * P.sq[1] + 1) / 2);  // FP32 operands of site 1
  }
  if (wc > kIntMax || P.L.maxcore > kIntMax || zt_cap > kIntMax || zw_cap > kIntMax || zf_cap > kIntMax)
    return TNR_ERANGE;
  const int64_t gram_cap = std::max<int64_t>(1, (P.d - 1) * 1024);
  if (bp) {
    memset(bp, 0, sizeof(*bp));
    bp->d0 = A.d;
    bp->m = P.m;
    bp->d = P.d;
    bp->K = (int)K;
    bp->k = pr.k;
    bp->q = pr.q;
    bp->mixed = mixed ? 1 : 0;
    bp->zip = zip ? 1 : 0;
    bp->status = 0;
    bp->seed = pr.seed;
    bp->tol = pr.opts.tol;
    bp->max_rank = pr.opts.max_rank;
    for (int k = 0; k < A.d; ++k) {
      bp->Ain[k] = A.core[k];
      bp->AI[k] = (int)A.I[k];
      bp->AJ[k] = (int)A.J[k];
    }
    for (int k = 0; k <= A.d; ++k) bp->AR[k] = (int)A.R[k];
    for (int k = 0; k < P.d; ++k) {
      bp->I[k] = (int)P.I[k];
      bp->J[k] = (int)P.J[k];
    }
    for (int k = 0; k <= P.d; ++k) bp->RA[k] = (int)P.RA[k];
    // Ain[] holds the merged operator's sites 1.. at index m-1+k, as the kernel reads them
    for (int k = 0; k < P.d; ++k) {
      bp->Uc[k] = pr.U->core[k];
      bp->Vc[k] = pr.V->core[k];
      bp->Ucap[k] = pr.U->cap[k];
      bp->Vcap[k] = pr.V->cap[k];
      if (!bp->Uc[k] || !bp->Vc[k]) return TNR_EINVAL;
    }
    bp->Sout = pr.S;
    bp->work_cap = wc;
    bp->gram_cap = gram_cap;
  }
  // scratch
  double *merged = nullptr, *merge_tmp = nullptr;
  if (P.m > 1) {
    merged = ar.take<double>(P.merged_elems);
    merge_tmp = ar.take<double>(P.merged_elems);
  }
  double *omega = ar.take<double>(P.omega_len);
  double *P0[TNR_MAX_SITES], *P1[TNR_MAX_SITES];
  for (int k = 0; k < P.d; ++k) P0[k] = ar.take<double>(P.pcap[k]);
  for (int k = 0; k < P.d; ++k) P1[k] = ar.take<double>(P.pcap[k]);
  double *tmp = ar.take<double>(P.L.maxcore);
  double *rbuf = ar.take<double>(P.L.maxbond * P.L.maxbond);
  double *work = ar.take<double>(wc);
  double *gram = ar.take<double>(gram_cap);
  double *Rm = ar.take<double>(K * K), *W = ar.take<double>(K * K), *Zr = ar.take<double>(K * K);
  double *Sv = ar.take<double>(K);
  double *zc0 = nullptr, *zc1 = nullptr, *zw = nullptr, *zt = nullptr;
  float *zf = nullptr;
  if (zip) {
    zc0 = ar.take<double>(zc_cap);
    zc1 = ar.take<double>(zc_cap);
    zw = ar.take<double>(zw_cap);
    zt = ar.take<double>(zt_cap);
    if (mixed) zf = ar.take<float>(zf_cap);
  }
  if (bp) {
    bp->zc[0] = zc0;
    bp->zc[1] = zc1;
    bp->zw = zw;
    bp->zt = zt;
    bp->zf = zf;
    bp->zc_cap = zc_cap;
    bp->zw_cap = zw_cap;
    bp->zt_cap = zt_cap;
    bp->zf_cap = mixed ? zf_cap : 0;
  }
  if (bp) {
    bp->merged = merged;
    bp->merge_tmp = merge_tmp;
    bp->omega = omega;
    for (int k = 0; k < P.d; ++k) {
      bp->P0[k] = P0[k];
      bp->P1[k] = P1[k];
      bp->pcap[k] = P.pcap[k];
    }
    bp->tmp = tmp;
    bp->rbuf = rbuf;
    bp->work = work;
    bp->gram = gram;
    bp->Rm = Rm;
    bp->W = W;
    bp->Zr = Zr;
    bp->Sv = Sv;
  }
  if (cost) {
    double c = 0.0;
    if (zip) {  // per product: the two contraction stages and the SVD step of every site
      for (int k = 1; k < P.d; ++k) {
        const double X = (double)std::max(P.I[k], P.J[k]), rows = (double)P.RA[k] * P.sq[k], w = X * zq[k + 1];
        const double n = std::min(rows, w);
        c += 2.0 * X * (double)P.sq[k] * P.RA[k + 1] * zq[k + 1] * P.sq[k + 1] + 2.0 * rows * w * X * P.RA[k + 1] +
             2.0 * std::max(rows, w) * n * n;
      }
      c += 2.0 * (double)std::max(P.I[0], P.J[0]) * K * P.RA[1] * zq[1] * (P.sq[1] + P.I[0]);
    } else {
      for (int k = 0; k < P.d; ++k) c += (double)P.pcap[k];
    }
    *cost = c * (2.0 * pr.q + 2.0);
  }
  if (bucket) *bucket = pow2_ceil(P.L.maxbond) * 4096 + pow2_ceil(std::max(P.I[0], P.J[0])) * 64 + pow2_ceil(K);
  return TNR_OK;
}

constexpr size_t kHeaderBytes = 256;  // queue counter

struct BatchHandle {
  int n = 0;
  tnr_problem *probs = nullptr;
  std::vector<int> order;  // queue position -> problem index
  BatchProblem *dprob = nullptr;
  int *dqueue = nullptr;
  std::vector<BatchProblem> host;  // descriptors as uploaded (results come back into a copy)
  int grid = 0, per_sm = 1;
  size_t smem = 0;
  int64_t bucket = 0;
  cudaGraphExec_t exec = nullptr;
};

// Dynamic shared memory per CTA for `per_sm` CTAs per SM.
size_t smem_for(int per_sm) {
  int dev = 0, max_optin = 0, per_mp = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_mp, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, (const void *)k_batch_solve);
  // 1 KB per CTA reserved by the system, the kernel's static shared memory
  int64_t each = (int64_t)per_mp / per_sm - 1024 - (int64_t)fa.sharedSizeBytes;
  each = std::min<int64_t>(each, (int64_t)max_optin - (int64_t)fa.sharedSizeBytes);
  each = (each / 1024) * 1024;
  return each > 0 ? (size_t)each : 0;
}

int configure(BatchHandle &h, int per_sm) {
  int dev = 0, sms = 0;
  TNR_CK(cudaGetDevice(&dev));
  TNR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  size_t smem = smem_for(per_sm);
  if (smem < 16 * 1024) return TNR_EINVAL;
  TNR_TRY(ensure_dynamic_smem((const void *)k_batch_solve, smem));
  int fit = 0;
  TNR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_batch_solve, kBT, smem));
  if (fit < 1) return TNR_EINVAL;
  h.per_sm = std::min(per_sm, fit);
  h.smem = smem;
  h.grid = std::max(1, std::min(h.n, sms * h.per_sm));
  return TNR_OK;
}

// Queue reset and the persistent kernel. record: count the launch (not while it is being
// captured into a graph; the graph launch is counted instead).
int launch(const BatchHandle &h, cudaStream_t s, bool record = true) {
  TNR_CK(cudaMemsetAsync(h.dqueue, 0, sizeof(int), s));
  if (record) stats_begin(K_BATCH, s);
  k_batch_solve<<<h.grid, kBT, h.smem, s>>>(h.dprob, h.n, h.dqueue, (int64_t)(h.smem / sizeof(double)));
  if (record) stats_end(K_BATCH, s);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// Autotuner: CTAs per SM for a shape bucket, chosen once per process by timing the batch.
std::mutex g_tune_mu;
std::map<int64_t, int> g_tuned;

int autotune(BatchHandle &h, cudaStream_t s) {
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tuned.find(h.bucket);
    if (it != g_tuned.end()) return configure(h, it->second);
  }
  cudaEvent_t a = nullptr, b = nullptr;
  TNR_CK(cudaEventCreate(&a));
  TNR_CK(cudaEventCreate(&b));
  int best = 1;
  float best_ms = 1e30f;
  int rc = TNR_OK;
  bool warmed = false;
  for (int per_sm : {1, 2, 3, 4}) {
    if (configure(h, per_sm) != TNR_OK || h.per_sm != per_sm) continue;
    if (!warmed) {  // module load, first-touch of the scratch
      rc = launch(h, s);
      if (rc != TNR_OK) break;
      warmed = true;
    }
    cudaEventRecord(a, s);
    rc = launch(h, s);
    if (rc != TNR_OK) break;
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      rc = TNR_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best_ms) {
      best_ms = ms;
      best = per_sm;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  TNR_TRY(rc);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned[h.bucket] = best;
  }
  return configure(h, best);
}

}  // namespace
}  // namespace tnr

using namespace tnr;

extern "C" int tnr_batch_workspace(int32_t n, const tnr_problem *probs, size_t *bytes) {
  if (n < 0 || (n > 0 && !probs) || !bytes) return TNR_EINVAL;
  Arena ar;
  ar.take<char>(kHeaderBytes);
  ar.take<BatchProblem>((size_t)std::max(n, 1));
  for (int32_t i = 0; i < n; ++i) TNR_TRY(plan_problem(probs[i], ar, nullptr, nullptr, nullptr));
  *bytes = ar.off;
  return TNR_OK;
}

extern "C" int tnr_batch_create(int32_t n, tnr_problem *probs, int32_t flags, void *ws, size_t ws_bytes, void *stream,
                                void **handle) {
  if (!handle) return TNR_EINVAL;
  *handle = nullptr;
  if (n < 1 || !probs || !ws || (flags & ~0xF3)) return TNR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BatchHandle *h = new (std::nothrow) BatchHandle;
  if (!h) return TNR_ENOMEM;
  h->n = n;
  h->probs = probs;
  h->host.resize(n);
  Arena ar;
  ar.base = static_cast<char *>(ws);
  ar.size = ws_bytes;
  h->dqueue = ar.take<int>(kHeaderBytes / sizeof(int));
  h->dprob = ar.take<BatchProblem>((size_t)n);
  std::vector<double> cost(n);
  std::vector<BatchProblem> plan(n);
  int64_t bucket = 0;
  for (int32_t i = 0; i < n; ++i) {
    probs[i].status = TNR_OK;
    int64_t b = 0;
    const int rc = plan_problem(probs[i], ar, &plan[i], &cost[i], &b);
    if (rc != TNR_OK || !ar.ok) {
      delete h;
      return rc != TNR_OK ? rc : TNR_ENOMEM;
    }
    bucket = std::max(bucket, b);
  }
  // queue order: decreasing estimated cost (longest first balances the persistent CTAs)
  h->order.resize(n);
  for (int32_t i = 0; i < n; ++i) h->order[i] = i;
  std::stable_sort(h->order.begin(), h->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (int32_t i = 0; i < n; ++i) h->host[i] = plan[h->order[i]];
  h->bucket = bucket;
  int rc = check_cuda_at(
      cudaMemcpyAsync(h->dprob, h->host.data(), sizeof(BatchProblem) * n, cudaMemcpyHostToDevice, s), __FILE__,
      __LINE__);
  if (rc == TNR_OK) rc = check_cuda_at(cudaStreamSynchronize(s), __FILE__, __LINE__);
  const int forced = (flags >> 4) & 15;  // CTAs per SM chosen by the caller
  if (rc == TNR_OK) rc = forced ? configure(*h, forced) : (flags & 1) ? autotune(*h, s) : configure(*h, 1);
  if (rc == TNR_OK && (flags & 2)) {  // capture the launch (queue reset + kernel) in a CUDA graph
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    rc = check_cuda_at(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), __FILE__, __LINE__);
    if (rc == TNR_OK) {
      rc = check_cuda_at(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), __FILE__, __LINE__);
      if (rc == TNR_OK) {
        const int lr = launch(*h, cs, false);
        const int er = check_cuda_at(cudaStreamEndCapture(cs, &g), __FILE__, __LINE__);
        rc = lr != TNR_OK ? lr : er;
      }
      if (rc == TNR_OK) rc = check_cuda_at(cudaGraphInstantiate(&h->exec, g, 0), __FILE__, __LINE__);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
    }
  }
  if (rc != TNR_OK) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    delete h;
    return rc;
  }
  *handle = h;
  return TNR_OK;
}

extern "C" int tnr_batch_launch(void *handle, void *stream) {
  if (!handle) return TNR_EINVAL;
  BatchHandle &h = *static_cast<BatchHandle *>(handle);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h.exec) {
    LaunchScope ls(K_BATCH, s);
    return check_cuda_at(cudaGraphLaunch(h.exec, s), __FILE__, __LINE__);
  }
  return launch(h, s);
}

extern "C" int tnr_batch_collect(void *handle, void *stream) {
  if (!handle) return TNR_EINVAL;
  BatchHandle &h = *static_cast<BatchHandle *>(handle);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<BatchProblem> res(h.n);
  TNR_CK(cudaMemcpyAsync(res.data(), h.dprob, sizeof(BatchProblem) * h.n, cudaMemcpyDeviceToHost, s));
  TNR_CK(cudaStreamSynchronize(s));
  int first = TNR_OK;
  double flops = 0.0;
  for (int i = 0; i < h.n; ++i) {
    const BatchProblem &r = res[i];
    flops += r.status == TNR_OK ? r.flops : 0.0;
    tnr_problem &pr = h.probs[h.order[i]];
    pr.status = r.status;
    if (r.status == TNR_OK) {
      const int d = r.d;
      tnr_mpo *U = pr.U, *V = pr.V;
      U->d = d;
      V->d = d;
      for (int k = 0; k < d; ++k) {
        U->I[k] = r.I[k];
        V->I[k] = r.J[k];
        U->J[k] = k == 0 ? r.k : 1;
        V->J[k] = k == 0 ? r.k : 1;
      }
      for (int k = 0; k <= d; ++k) {
        U->R[k] = r.RU[k];
        V->R[k] = r.RV[k];
      }
    } else if (first == TNR_OK) {
      first = r.status;
    }
  }
  stats_work(K_BATCH, flops);  // algorithmic FP64 flops of one launch of the batch
  return first;
}

extern "C" int tnr_batch_destroy(void *handle) {
  if (!handle) return TNR_OK;
  BatchHandle *h = static_cast<BatchHandle *>(handle);
  if (h->exec) cudaGraphExecDestroy(h->exec);
  delete h;
  return TNR_OK;
}

extern "C" int tnr_batch_config(void *handle, int32_t *grid, int32_t *ctas_per_sm, int64_t *smem_bytes) {
  if (!handle) return TNR_EINVAL;
  const BatchHandle &h = *static_cast<const BatchHandle *>(handle);
  if (grid) *grid = h.grid;
  if (ctas_per_sm) *ctas_per_sm = h.per_sm;
  if (smem_bytes) *smem_bytes = (int64_t)h.smem;
  return TNR_OK;
}
