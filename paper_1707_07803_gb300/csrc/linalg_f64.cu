// FP64 dense building blocks for the MPO sweeps: batched GEMM, thin Householder QR spread
// over many CTAs, one-sided Jacobi SVD, and small copy kernels. All matrices column-major.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate (roughly 7 GFLOP/s per SM), so every FP64
// kernel here is written to spread its arithmetic over as many SMs as the problem allows:
// the GEMM picks tile sizes (and split-K) that give at least two CTAs per SM, and the QR
// distributes columns over CTAs that exchange Householder vectors through L2 with
// release/acquire flags, so that its sequential chain of reflectors costs one flag hop per
// column rather than a full trailing update on one SM.
#include <cfloat>
#include <cmath>
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "dev_common.cuh"
#include "jacobi.cuh"
#include "tnr_internal.cuh"
#include "qr_tpc.cuh"

namespace tnr {
namespace {

// ------------------------------------------------------------------------------------------
// GEMM: C[b] = alpha op(A[b]) op(B[b]) + beta C[b].
// ------------------------------------------------------------------------------------------
template <int BM, int BN, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int64_t m, int64_t n, int64_t k, double alpha,
                                              const double *__restrict__ A, int64_t lda, int64_t sa,
                                              const double *__restrict__ B, int64_t ldb, int64_t sb, double beta,
                                              double *__restrict__ C, int64_t ldc, int64_t sc, int splits,
                                              int64_t kchunk) {
  constexpr int BK = 16;
  constexpr int TMr = BM / 16, TNr = BN / 16;  // micro-tile per thread
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int batch = blockIdx.z / splits, split = blockIdx.z % splits;
  A += batch * sa;
  B += batch * sb;
  C += batch * sc;
  const int64_t row0 = (int64_t)blockIdx.x * BM, col0 = (int64_t)blockIdx.y * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[TMr][TNr];
#pragma unroll
  for (int i = 0; i < TMr; ++i)
#pragma unroll
    for (int j = 0; j < TNr; ++j) acc[i][j] = 0.0;
  const int64_t kbeg = split * kchunk;
  const int64_t kend = min(k, kbeg + kchunk);
  for (int64_t kk = kbeg; kk < kend; kk += BK) {
    for (int idx = threadIdx.x; idx < BK * BM; idx += 256) {
      const int l = TA ? idx % BK : idx / BM;
      const int i = TA ? idx / BK : idx % BM;
      const int64_t gi = row0 + i, gk = kk + l;
      double v = 0.0;
      if (gi < m && gk < kend) v = TA ? A[gk + lda * gi] : A[gi + lda * gk];
      As[l][i] = v;
    }
    for (int idx = threadIdx.x; idx < BK * BN; idx += 256) {
      const int l = TB ? idx / BN : idx % BK;
      const int j = TB ? idx % BN : idx / BK;
      const int64_t gj = col0 + j, gk = kk + l;
      double v = 0.0;
      if (gj < n && gk < kend) v = TB ? B[gj + ldb * gk] : B[gk + ldb * gj];
      Bs[l][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < BK; ++l) {
      double a[TMr], b[TNr];
#pragma unroll
      for (int i = 0; i < TMr; ++i) a[i] = As[l][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < TNr; ++j) b[j] = Bs[l][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < TMr; ++i)
#pragma unroll
        for (int j = 0; j < TNr; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TMr; ++i) {
    const int64_t gi = row0 + tx + 16 * i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < TNr; ++j) {
      const int64_t gj = col0 + ty + 16 * j;
      if (gj >= n) continue;
      double *c = C + gi + ldc * gj;
      if (splits > 1)
        atomicAdd(c, alpha * acc[i][j]);
      else
        *c = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *c);
    }
  }
}

__global__ void k_scale_matrix(double *C, int64_t ldc, int64_t sc, int m, int n, double beta) {
  const int64_t b = blockIdx.z;
  const unsigned mn = (unsigned)m * (unsigned)n;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mn; idx += gridDim.x * blockDim.x) {
    double *c = C + b * sc + (idx % (unsigned)m) + ldc * (idx / (unsigned)m);
    *c = beta == 0.0 ? 0.0 : beta * *c;
  }
}

// Small NN products (m n <= 64K outputs, k <= 1024): one thread per output, four independent
// accumulators so the 64-cycle FP64 FMA latency overlaps; no staging or barriers.
__global__ void __launch_bounds__(256) k_gemm_tiny(int m, int n, int k, double alpha, const double *__restrict__ A,
                                                   int64_t lda, int64_t sa, const double *__restrict__ B, int64_t ldb,
                                                   int64_t sb, double beta, double *__restrict__ C, int64_t ldc,
                                                   int64_t sc) {
  const unsigned mn = (unsigned)m * (unsigned)n;
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mn) return;
  const int64_t b = blockIdx.y;
  const unsigned i = idx % (unsigned)m, j = idx / (unsigned)m;
  const double *a = A + b * sa + i;
  const double *bb = B + b * sb + ldb * j;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int l = 0;
  for (; l + 3 < k; l += 4) {
    s0 = fma(a[lda * l], bb[l], s0);
    s1 = fma(a[lda * (l + 1)], bb[l + 1], s1);
    s2 = fma(a[lda * (l + 2)], bb[l + 2], s2);
    s3 = fma(a[lda * (l + 3)], bb[l + 3], s3);
  }
  for (; l < k; ++l) s0 = fma(a[lda * l], bb[l], s0);
  double *c = C + b * sc + i + ldc * j;
  const double v = alpha * ((s0 + s1) + (s2 + s3));
  *c = beta == 0.0 ? v : fma(beta, *c, v);
}

template <int BM, int BN>
int launch_gemm(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double *A,
                int64_t lda, int64_t sa, const double *B, int64_t ldb, int64_t sb, double beta, double *C, int64_t ldc,
                int64_t sc, int64_t batch, int splits) {
  const int64_t kchunk = cdiv(cdiv(k, splits), 16) * 16;
  splits = (int)cdiv(k, kchunk);
  dim3 grid((unsigned)cdiv(m, BM), (unsigned)cdiv(n, BN), (unsigned)(batch * splits));
  if (splits > 1) {
    LaunchScope ls(K_GEMM, s);
    k_scale_matrix<<<dim3(64, 1, (unsigned)batch), 256, 0, s>>>(C, ldc, sc, (int)m, (int)n, beta);
  }
  LaunchScope ls(K_GEMM, s);
#define TNR_G(TA_, TB_) \
  k_gemm<BM, BN, TA_, TB_><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc, splits, kchunk)
  if (!ta && !tb) TNR_G(false, false);
  else if (ta && !tb) TNR_G(true, false);
  else if (!ta && tb) TNR_G(false, true);
  else TNR_G(true, true);
#undef TNR_G
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// ------------------------------------------------------------------------------------------
// Block reductions (256 threads).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // protect red from a previous use
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) t += red[w];
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool qr_wait_flag(const unsigned *f, int *status) {
  long long spins = 0;
  while (ld_acquire(f) == 0u) {
    if (++spins > kSpinCap) {
      set_status(status, TNR_ETIMEOUT);
      return false;
    }
  }
  return true;
}

// ------------------------------------------------------------------------------------------
// Householder QR, one warp per CTA, columns distributed cyclically over P CTAs (cooperative
// launch, so all CTAs are resident; P <= #SMs so every CTA has an SM's FP64 pipe to itself).
// Reflector j (LAPACK dlarfg convention: beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
// v = x / (alpha - beta), v_j = 1) is computed by the owner of column j, written to V[:, j]
// and published with a release store to flags[j]; every CTA applies it to its own columns
// after an acquire load. The owner of column j+1 applies reflector j to column j+1 first and
// publishes reflector j+1 before updating its other columns (one-column lookahead), so the
// critical path per column is one flag hop plus one column update. A single warp per CTA
// keeps the FP64 instruction count of each reduction at 5 shuffle-adds (FP64 issue, not
// bandwidth, limits these small reductions on GB300). Waits are bounded (kSpinCap polls); on
// timeout the kernel records TNR_ETIMEOUT and returns.
// ------------------------------------------------------------------------------------------
struct QrArgs {
  double *A;
  int64_t m, n, lda;
  double *R;
  int64_t ldr;
  double *V;  // m x nref (ld m)
  double *tau;
  unsigned *flags;
  int *status;
};

__device__ __forceinline__ bool qr_wait(const QrArgs &a, int64_t j) {
  long long spins = 0;
  while (ld_acquire(a.flags + j) == 0u) {
    if (++spins > kSpinCap) {
      set_status(a.status, TNR_ETIMEOUT);
      return false;
    }
  }
  return true;
}

// The CTA's own columns live in shared memory for the whole factorisation (cols, nc x m);
// only reflectors travel through L2.
__device__ void qr_make_reflector(const QrArgs &a, double *col, int64_t j) {
  const int lane = threadIdx.x;
  double sig = 0.0;
  for (int64_t i = j + 1 + lane; i < a.m; i += 32) sig = fma(col[i], col[i], sig);
  sig = warp_sum(sig);
  const double alpha = col[j];
  double tau = 0.0, beta = alpha, scal = 0.0;
  if (sig > 0.0) {
    householder_params(alpha, sig, beta, tau, scal);
  }
  double *v = a.V + a.m * j;
  for (int64_t i = j + 1 + lane; i < a.m; i += 32) {
    const double x = col[i] * scal;
    v[i] = x;
    col[i] = x;  // keep v below the diagonal of the cached column
  }
  if (lane == 0) {
    v[j] = 1.0;
    col[j] = beta;
    a.tau[j] = tau;
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release(a.flags + j, 1u);
}

// Apply H_j = I - tau v v^T (v in vs, rows j..m-1) to a cached column.
__device__ __forceinline__ void qr_apply(const QrArgs &a, const double *vs, double tau, int64_t j, double *col) {
  const int lane = threadIdx.x;
  double w0 = 0.0, w1 = 0.0;
  int64_t i = j + lane;
  for (; i + 32 < a.m; i += 64) {
    w0 = fma(vs[i - j], col[i], w0);
    w1 = fma(vs[i + 32 - j], col[i + 32], w1);
  }
  if (i < a.m) w0 = fma(vs[i - j], col[i], w0);
  const double w = warp_sum(w0 + w1) * tau;
  for (int64_t t = j + lane; t < a.m; t += 32) col[t] = fma(-w, vs[t - j], col[t]);
  __syncwarp();
}

// Load rows j..m-1 of reflector j from L2 with all loads in flight before the stores.
__device__ __forceinline__ void qr_load_reflector(const QrArgs &a, int64_t j, double *vs) {
  const int lane = threadIdx.x;
  const double *src = a.V + a.m * j;
  int64_t i = j + lane;
  for (; i + 96 < a.m; i += 128) {
    const double x0 = __ldcg(src + i), x1 = __ldcg(src + i + 32), x2 = __ldcg(src + i + 64),
                 x3 = __ldcg(src + i + 96);
    vs[i - j] = x0;
    vs[i + 32 - j] = x1;
    vs[i + 64 - j] = x2;
    vs[i + 96 - j] = x3;
  }
  for (; i < a.m; i += 32) vs[i - j] = __ldcg(src + i);
}

__global__ void __launch_bounds__(32) k_qr_coop(QrArgs a) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x;
  const int64_t P = gridDim.x, c = blockIdx.x;
  const int64_t m = a.m;
  const int64_t nref = m < a.n ? m : a.n;
  const int64_t nc = (a.n - c + P - 1) / P;  // my columns l = c + q P
  double *cols = sm;                         // nc x m
  double *vs = sm + nc * m;                  // m
  for (int64_t q = 0; q < nc; ++q) {
    const double *src = a.A + a.lda * (c + q * P);
    for (int64_t i = lane; i < m; i += 32) cols[q * m + i] = src[i];
  }
  __syncwarp();
  if (c == 0 && nref > 0) qr_make_reflector(a, cols, 0);
  for (int64_t j = 0; j < nref; ++j) {
    const int64_t l0 = j + 1 + ((c - (j + 1) % P) + P) % P;  // my first column > j
    if (l0 >= a.n) break;  // owned columns only move right: nothing left to update
    if (!qr_wait(a, j)) return;
    qr_load_reflector(a, j, vs);
    const double tau = __ldcg(a.tau + j);
    __syncwarp();
    for (int64_t l = l0; l < a.n; l += P) {
      double *col = cols + ((l - c) / P) * m;
      if (tau != 0.0) qr_apply(a, vs, tau, j, col);
      if (l == j + 1 && l < nref) qr_make_reflector(a, col, l);
    }
    __syncwarp();
  }
  // R: column l of the upper trapezoid (rows 0..min(l, nref-1)), zeros below.
  for (int64_t q = 0; q < nc; ++q) {
    const int64_t l = c + q * P;
    for (int64_t i = lane; i < nref; i += 32) a.R[i + a.ldr * l] = i <= l ? cols[q * m + i] : 0.0;
  }
  __syncwarp();
  // Explicit Q, column l = H_0 ... H_l e_l for my columns l < nref. Every reflector j <= l
  // was acquired above (the owner of l waited for each j < l and made l itself).
  for (int64_t q = 0; q < nc; ++q) {
    const int64_t l = c + q * P;
    if (l >= nref) break;
    double *qv = cols + q * m;  // reuse the cached column
    for (int64_t i = lane; i < m; i += 32) qv[i] = (i == l) ? 1.0 : 0.0;
    __syncwarp();
    for (int64_t j = l; j >= 0; --j) {
      const double tau = __ldcg(a.tau + j);
      if (tau == 0.0) continue;
      qr_load_reflector(a, j, vs);
      __syncwarp();
      double w0 = 0.0, w1 = 0.0;
      int64_t i = j + lane;
      for (; i + 32 < m; i += 64) {
        w0 = fma(vs[i - j], qv[i], w0);
        w1 = fma(vs[i + 32 - j], qv[i + 32], w1);
      }
      if (i < m) w0 = fma(vs[i - j], qv[i], w0);
      const double w = warp_sum(w0 + w1) * tau;
      for (int64_t t = j + lane; t < m; t += 32) qv[t] = fma(-w, vs[t - j], qv[t]);
      __syncwarp();
    }
    double *dst = a.A + a.lda * l;
    for (int64_t i = lane; i < m; i += 32) dst[i] = qv[i];
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// Column-pivoted Householder QR with a noise-level cutoff (rank-revealing), for the
// left-to-right orthogonalisation sweep. M (m x n) = Q R + E with Q (m x r) orthonormal,
// R = Q^T M (r x n, original column order) and every column of E below the cutoff
// c * ||M||_F. The discarded directions are of the size of the backward error of an
// unpivoted Householder QR of M (a few n eps ||M||_F), so they are the directions the
// rounding sweep that follows must remove anyway; the bond shrinks to the numerical rank of
// M right away instead of after a full-width factorisation and SVD.
//
// One warp per CTA, P <= #SMs CTAs, each caching its columns (l = c mod P) in shared memory.
// Step i: every CTA proposes its largest remaining column norm through a 64-bit atomicMax
// (high bits of the double, low 20 bits the complemented column index, so ties pick the
// lowest column) and arrives on a per-step counter; once all P have arrived, the owner of the
// pivot builds reflector i (dlarfg convention), publishes it (release flag), and every CTA
// applies it to its unpivoted columns and recomputes their norms over rows > i exactly.
// The sweep stops when the largest remaining norm is at or below the cutoff; r >= 1.
// All waits are bounded; a timeout sets TNR_ETIMEOUT and the kernel returns.
// ------------------------------------------------------------------------------------------
struct QrcpArgs {
  double *A;
  int64_t m, n, lda;
  double *R;  // r x n, ld ldr (ldr >= min(m, n))
  int64_t ldr;
  double *V;  // m x nref
  double *tau;
  unsigned long long *best;  // nref
  unsigned *cnt;             // nref + 1
  unsigned *flags;           // nref
  double *fro2;              // 1
  int64_t *r_out;            // device rank
  double cut_rel;
  int *status;
};

__device__ __forceinline__ bool wait_count(const unsigned *p, unsigned target, int *status) {
  long long spins = 0;
  while (ld_acquire(p) < target) {
    if (++spins > kSpinCap) {
      set_status(status, TNR_ETIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void arrive(unsigned *p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

__global__ void __launch_bounds__(32) k_qrcp(QrcpArgs a) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x;
  const int64_t P = gridDim.x, c = blockIdx.x;
  const int64_t m = a.m, n = a.n;
  const int64_t nref = m < n ? m : n;
  const int64_t nc = (n - c + P - 1) / P;  // number of my columns
  double *cols = sm;                       // nc x m
  double *vs = sm + nc * m;                // m
  double *nrm = vs + m;                    // nc
  int *piv = reinterpret_cast<int *>(nrm + nc);  // nc: 1 when pivoted
  // load my columns and their norms
  double mine = 0.0;
  for (int64_t q = 0; q < nc; ++q) {
    const double *src = a.A + a.lda * (c + q * P);
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) {
      const double x = src[i];
      cols[q * m + i] = x;
      s = fma(x, x, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      nrm[q] = s;
      piv[q] = 0;
    }
    mine += s;
  }
  __syncwarp();
  if (lane == 0) {
    atomicAdd(a.fro2, mine);
    __threadfence();
    arrive(a.cnt + 0);
  }
  if (!wait_count(a.cnt + 0, (unsigned)P, a.status)) return;
  const double cut2 = a.cut_rel * a.cut_rel * __ldcg(a.fro2);
  int64_t r = 0;
  for (int64_t i = 0; i < nref; ++i) {
    // propose my best remaining column
    unsigned long long key = 0ull;
    for (int64_t q = 0; q < nc; ++q) {
      if (piv[q]) continue;
      const double v2 = nrm[q];
      const unsigned long long k2 = (__double_as_longlong(v2 > 0.0 ? v2 : 0.0) & ~0xFFFFFull) |
                                    (unsigned long long)(0xFFFFF - (c + q * P));
      if (k2 > key) key = k2;
    }
    if (lane == 0) {
      if (key) atomicMax(a.best + i, key);
      __threadfence();
      arrive(a.cnt + i + 1);
    }
    if (!wait_count(a.cnt + i + 1, (unsigned)P, a.status)) return;
    const unsigned long long b = __ldcg(a.best + i);
    // every unpivoted column contributes a nonzero key (its complemented index), so b != 0
    if (b == 0ull) break;
    const double bn2 = __longlong_as_double((long long)(b & ~0xFFFFFull));
    const int64_t p = 0xFFFFF - (int64_t)(b & 0xFFFFFull);
    if (i > 0 && bn2 <= cut2) break;  // remaining columns are noise (keep r >= 1)
    r = i + 1;
    if (p % P == c) {  // I own the pivot: build reflector i from rows i..m-1 of column p
      const int64_t q = p / P;
      double *col = cols + q * m;
      double sig = 0.0;
      for (int64_t t = i + 1 + lane; t < m; t += 32) sig = fma(col[t], col[t], sig);
      sig = warp_sum(sig);
      const double alpha = col[i];
      double tau = 0.0, beta = alpha, scal = 0.0;
      if (sig > 0.0) {
        householder_params(alpha, sig, beta, tau, scal);
      }
      double *v = a.V + m * i;
      for (int64_t t = i + 1 + lane; t < m; t += 32) {
        v[t] = col[t] * scal;
        col[t] = 0.0;
      }
      if (lane == 0) {
        v[i] = 1.0;
        col[i] = beta;
        a.tau[i] = tau;
        piv[q] = 1;
        nrm[q] = 0.0;
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(a.flags + i, 1u);
    }
    // apply reflector i to my unpivoted columns
    bool any = false;
    for (int64_t q = 0; q < nc; ++q) any |= !piv[q];
    if (!any) continue;
    if (!qr_wait_flag(a.flags + i, a.status)) return;
    for (int64_t t = i + lane; t < m; t += 32) vs[t - i] = __ldcg(a.V + m * i + t);
    const double tau = __ldcg(a.tau + i);
    __syncwarp();
    for (int64_t q = 0; q < nc; ++q) {
      if (piv[q]) continue;
      double *col = cols + q * m;
      if (tau != 0.0) {
        double w = 0.0;
        for (int64_t t = i + lane; t < m; t += 32) w = fma(vs[t - i], col[t], w);
        w = warp_sum(w) * tau;
        for (int64_t t = i + lane; t < m; t += 32) col[t] = fma(-w, vs[t - i], col[t]);
      }
      double s = 0.0;
      for (int64_t t = i + 1 + lane; t < m; t += 32) s = fma(col[t], col[t], s);
      s = warp_sum(s);
      if (lane == 0) nrm[q] = s;
    }
    __syncwarp();
  }
  if (c == 0 && lane == 0) *a.r_out = r;
  // R = rows 0..r-1 of every column (original order)
  for (int64_t q = 0; q < nc; ++q) {
    const int64_t l = c + q * P;
    for (int64_t t = lane; t < r; t += 32) a.R[t + a.ldr * l] = cols[q * m + t];
  }
  // Explicit Q (m x r): column l = H_0 ... H_l e_l, in place of A. All CTAs loaded their
  // columns before the first step's counter completed, so overwriting A is safe here.
  for (int64_t l = c; l < r; l += P) {
    double *qv = vs;  // reuse as the working column
    for (int64_t t = lane; t < m; t += 32) qv[t] = (t == l) ? 1.0 : 0.0;
    __syncwarp();
    for (int64_t j = l; j >= 0; --j) {
      if (!qr_wait_flag(a.flags + j, a.status)) return;
      const double tau = __ldcg(a.tau + j);
      if (tau == 0.0) continue;
      const double *v = a.V + m * j;
      double w = 0.0;
      for (int64_t t = j + lane; t < m; t += 32) w = fma(__ldcg(v + t), qv[t], w);
      w = warp_sum(w) * tau;
      for (int64_t t = j + lane; t < m; t += 32) qv[t] = fma(-w, __ldcg(v + t), qv[t]);
      __syncwarp();
    }
    double *dst = a.A + a.lda * l;
    for (int64_t t = lane; t < m; t += 32) dst[t] = qv[t];
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// Householder QR of a small matrix in one CTA (whole matrix in shared memory), optionally
// column-pivoted with a noise-level cutoff. A = op(src) is m x n (op = transpose when
// trans_src). Unpivoted: A = Q R, r = min(m, n). Pivoted (dgeqp3-style, columns swapped
// physically): A P = Q R_p, stopping when the largest remaining column norm is at or below
// cut_rel ||A||_F (r >= 1). Outputs: Q (m x r) explicit, written as Q or Q^T (trans_q); and
// R = Q^T A in the ORIGINAL column order (r x n), written as R or R^T (trans_r); r to *r_out.
// Warps own columns, lanes own rows; FP64 reductions stay within one warp.
// ------------------------------------------------------------------------------------------


__global__ void __launch_bounds__(kSmallThreads) k_qr_small(QrSmallArgs a) {
  extern __shared__ double sm[];
  const int m = a.m, n = a.n;
  const int nref = m < n ? m : n;
  double *A = sm;               // m x n, ld m
  double *nrm = A + m * n;      // n
  double *tau = nrm + n;        // nref
  int *perm = reinterpret_cast<int *>(tau + nref);  // n
  __shared__ double s_red[32];
  __shared__ int s_idx[32];
  __shared__ int s_r;
  __shared__ double s_cut2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kSmallThreads / 32;
  for (int idx = threadIdx.x; idx < m * n; idx += kSmallThreads) {
    const int i = idx % m, j = idx / m;
    A[idx] = a.trans_src ? a.src[j + a.lds * i] : a.src[i + a.lds * j];
  }
  for (int j = threadIdx.x; j < n; j += kSmallThreads) perm[j] = (int)j;
  __syncthreads();
  // column norms
  for (int j = warp; j < n; j += NW) {
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s = fma(A[i + m * j], A[i + m * j], s);
    s = warp_sum(s);
    if (lane == 0) nrm[j] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int j = 0; j < n; ++j) f += nrm[j];
    s_cut2 = a.cut_rel * a.cut_rel * f;
    s_r = (int)nref;
  }
  __syncthreads();
  for (int i = 0; i < nref; ++i) {
    if (a.pivot) {
      // argmax of nrm[i..n-1] (lowest index on ties)
      double bv = -1.0;
      int bi = (int)i;
      for (int j = i + threadIdx.x; j < n; j += kSmallThreads) {
        if (nrm[j] > bv) {
          bv = nrm[j];
          bi = (int)j;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_red[warp] = bv;
        s_idx[warp] = bi;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double b = s_red[0];
        int bj = s_idx[0];
        for (int w = 1; w < NW; ++w)
          if (s_red[w] > b || (s_red[w] == b && s_idx[w] < bj)) {
            b = s_red[w];
            bj = s_idx[w];
          }
        s_idx[0] = bj;
        s_red[0] = b;
        if (i > 0 && b <= s_cut2) s_r = (int)i;
      }
      __syncthreads();
      if (s_r == (int)i) break;
      const int p = s_idx[0];
      if (p != i) {
        for (int t = threadIdx.x; t < m; t += kSmallThreads) {
          const double x = A[t + m * i];
          A[t + m * i] = A[t + m * p];
          A[t + m * p] = x;
        }
        if (threadIdx.x == 0) {
          const double x = nrm[i];
          nrm[i] = nrm[p];
          nrm[p] = x;
          const int q = perm[i];
          perm[i] = perm[p];
          perm[p] = q;
        }
      }
      __syncthreads();
    }
    // reflector from A[i:, i] (warp 0)
    if (warp == 0) {
      double *col = A + m * i;
      double sig = 0.0;
      for (int t = i + 1 + lane; t < m; t += 32) sig = fma(col[t], col[t], sig);
      sig = warp_sum(sig);
      const double alpha = col[i];
      double tv = 0.0, beta = alpha, scal = 0.0;
      if (sig > 0.0) {
        householder_params(alpha, sig, beta, tv, scal);
      }
      for (int t = i + 1 + lane; t < m; t += 32) col[t] *= scal;  // v below the diagonal
      __syncwarp();
      if (lane == 0) {
        col[i] = beta;
        tau[i] = tv;
      }
    }
    __syncthreads();
    // apply to columns j > i and refresh their norms over rows > i
    const double tv = tau[i];
    const double *v = A + m * i;
    for (int j = i + 1 + warp; j < n; j += NW) {
      double *col = A + m * j;
      if (tv != 0.0) {
        double w = lane == 0 ? col[i] : 0.0, w1 = 0.0;
        int t = i + 1 + lane;
        for (; t + 32 < m; t += 64) {
          w = fma(v[t], col[t], w);
          w1 = fma(v[t + 32], col[t + 32], w1);
        }
        if (t < m) w = fma(v[t], col[t], w);
        w = warp_sum(w + w1) * tv;
        if (lane == 0) col[i] -= w;
        for (int t = i + 1 + lane; t < m; t += 32) col[t] = fma(-w, v[t], col[t]);
      }
      if (a.pivot) {
        double s = 0.0;
        for (int t = i + 1 + lane; t < m; t += 32) s = fma(col[t], col[t], s);
        s = warp_sum(s);
        if (lane == 0) nrm[j] = s;
      }
    }
    __syncthreads();
  }
  const int r = s_r;
  if (threadIdx.x == 0 && a.r_out) *a.r_out = r;
  const int ldq = a.ldq > 0 ? a.ldq : r;  // ldq <= 0: Q^T packed with leading dimension r
  // R = rows 0..r-1 of the transformed matrix, upper trapezoid, scattered to original order
  for (int idx = threadIdx.x; idx < r * n; idx += kSmallThreads) {
    const int t = idx % r, j = idx / r;
    const double x = t <= j ? A[t + m * j] : 0.0;
    const int oj = perm[j];
    if (a.trans_r)
      a.R[oj + a.ldr * t] = x;
    else
      a.R[t + a.ldr * oj] = x;
  }
  __syncthreads();
  // Q = H_0 ... H_{r-1} [I_r; 0]: one warp per column, v_j read from below the diagonal
  for (int l = warp; l < r; l += NW) {
    // the column is accumulated directly in the output buffer
    double *q = a.trans_q ? nullptr : a.Q + ldq * l;
    // accumulate in a strided view: element t at qa(t)
    auto qa = [&](int t) -> double & { return a.trans_q ? a.Q[l + ldq * t] : q[t]; };
    for (int t = lane; t < m; t += 32) qa(t) = (t == l) ? 1.0 : 0.0;
    __syncwarp();
    for (int j = l; j >= 0; --j) {
      const double tj = tau[j];
      if (tj == 0.0) continue;
      const double *vj = A + m * j;
      double w = 0.0;
      for (int t = j + lane; t < m; t += 32) w = fma(t == j ? 1.0 : vj[t], qa(t), w);
      w = warp_sum(w) * tj;
      for (int t = j + lane; t < m; t += 32) qa(t) = fma(-w, t == j ? 1.0 : vj[t], qa(t));
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------------------------------
// Small QR for short columns (m <= 64): one thread owns one column and streams it alone, so no
// FP64 shuffle reductions are spent on columns shorter than a warp. The matrix is kept
// row-major in shared memory (consecutive threads touch consecutive words). Same contract and
// outputs as k_qr_small. Column pivoting uses norm downdating with the LAPACK (dgeqp3)
// safeguard: the norm of column j below row i is updated as ||.||^2 - R(i,j)^2 and recomputed
// when the downdate has lost more than half of its digits.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSmallThreads) k_qr_small_tpc(QrSmallArgs a) {
  extern __shared__ double sm[];
  qr_tpc_cta(a, sm);
}

// ------------------------------------------------------------------------------------------
// SVD of an n x n matrix G = U S V^T: one-sided (Hestenes) Jacobi sweeps in FP32 (jacobi.cuh:
// column pairs of a round-robin tournament rotated until every pair is orthogonal to FP32
// accuracy; columns at the rounding level of the whole matrix are not rotated), then the
// matrix-product refinement to FP64 accuracy when the FP32 singular values are separated, else
// Newton-Schulz and FP64 sweeps. Launched as one CTA, or, with the working set in shared memory
// and n <= 32, as a thread-block cluster whose CTA 0 runs the sweeps and whose CTAs share the
// refinement's products. Results sorted by descending singular value.
// ------------------------------------------------------------------------------------------
constexpr int kJacThreads = 512;

__global__ void __launch_bounds__(kJacThreads) k_jacobi(double *G, int n, int ldg, double *S, double *V, int ldv,
                                                        double *Gw, double *Vw, int *status) {
  extern __shared__ double sm[];
  __shared__ double s_norm[1024];
  __shared__ double s_inv[1024];
  const bool in_smem = Gw == nullptr;
  double *g = in_smem ? sm : Gw;          // working copy, ld n
  double *v = in_smem ? sm + n * n : Vw;  // working V, ld n
  double *jw = v + n * n;                 // work of the mixed-precision sweeps (after V)
  const int nthr = blockDim.x;
  for (int idx = threadIdx.x; idx < n * n; idx += nthr) {
    const int i = idx % n, j = idx / n;
    g[idx] = G[i + ldg * j];
    v[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // FP32 sweeps, then the product refinement (or, for close singular values, the FP64 sweeps)
  const unsigned nc = cluster_nctarank();  // 1: launched without a cluster
  if (nc == 1) {
    jacobi_sweeps_mixed(g, v, n, s_norm, jw, jw + jacobi_mixed_work(n));  // jacobi.cuh
  } else {
    // a cluster (working set in shared memory): CTA 0 runs the FP32 sweeps and stores V0 into
    // every CTA's work area, then all CTAs share the refinement's products; CTA 0 alone runs the
    // FP64 sweeps if the refinement declines, and writes the results
    const unsigned me = cluster_ctarank();
    const int np = n * (n + 1);
    double *v0 = jw + np;  // where jacobi_fp32_phase leaves V0 (ld n + 1)
    __shared__ int s_try;  // the refinement is worth trying (decided on CTA 0, stored into every CTA)
    if (me == 0) {
      jacobi_fp32_phase(g, n, s_norm, jw);
      const bool plausible = jacobi_refine_plausible(reinterpret_cast<const float *>(s_norm), n);
      if (plausible)
        for (int idx = threadIdx.x; idx < np; idx += nthr)
          for (unsigned rk = 1; rk < nc; ++rk) dsmem_st_f64(dsmem_addr(v0 + idx, rk), v0[idx]);
      if (threadIdx.x < (int)nc) dsmem_st_s32(dsmem_addr(&s_try, (unsigned)threadIdx.x), plausible ? 1 : 0);
    }
    cluster_sync_all();
    const bool ok = s_try && jacobi_refine(g, v0, n + 1, v, n, jw + jacobi_mixed_work(n), true);
    if (me != 0) return;  // no shared-memory access between CTAs follows the last cluster barrier
    if (!ok) jacobi_fp64_finish(g, v, n, s_norm, jw);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = nthr / 32;
  // final column norms and their reciprocals, one thread per column (the square roots and
  // divisions are FP64 instruction sequences: one per warp this way, not one per column)
  for (int j = threadIdx.x; j < n; j += nthr) {
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < n; i += 2) {
      s0 = fma(g[i + n * j], g[i + n * j], s0);
      s1 = fma(g[i + 1 + n * j], g[i + 1 + n * j], s1);
    }
    if (i < n) s0 = fma(g[i + n * j], g[i + n * j], s0);
    const double sj = sqrt(s0 + s1);
    s_norm[j] = sj;
    s_inv[j] = sj > 0.0 ? 1.0 / sj : 0.0;
  }
  __syncthreads();
  // rank of each column by descending norm (stable), then scatter.
  for (int j = warp; j < n; j += nw) {
    const double sj = s_norm[j];
    int rank = 0;
    for (int i = lane; i < n; i += 32) {
      const double si = s_norm[i];
      rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const double inv = s_inv[j];
    for (int i = lane; i < n; i += 32) {
      G[i + ldg * rank] = g[i + n * j] * inv;
      V[i + ldv * rank] = v[i + n * j];
    }
    if (lane == 0) S[rank] = sj;
  }
}

__global__ void k_copy(const double *__restrict__ src, int64_t lds, double *__restrict__ dst, int64_t ldd, int m, int n,
                       int transpose) {
  // dst (m x n) = src (m x n) or src^T (src is n x m when transposing); m * n < 2^31
  const unsigned mn = (unsigned)m * (unsigned)n;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mn; idx += gridDim.x * blockDim.x) {
    const unsigned i = idx % (unsigned)m, j = idx / (unsigned)m;
    dst[i + ldd * j] = transpose ? src[j + lds * i] : src[i + lds * j];
  }
}

__global__ void k_scale_cols(double *A, int64_t lda, int m, int n, const double *scale) {
  const unsigned mn = (unsigned)m * (unsigned)n;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mn; idx += gridDim.x * blockDim.x) {
    const unsigned i = idx % (unsigned)m, j = idx / (unsigned)m;
    A[i + lda * j] *= scale[j];
  }
}

int grid_for(int64_t work, int threads = 256) {
  int64_t g = cdiv(work, threads);
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

}  // namespace

int gemm_f64(cudaStream_t s, bool transA, bool transB, int64_t m, int64_t n, int64_t k, double alpha, const double *A,
             int64_t lda, int64_t sa, const double *B, int64_t ldb, int64_t sb, double beta, double *C, int64_t ldc,
             int64_t sc, int64_t batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return TNR_OK;
  if (k <= 0) {
    LaunchScope ls(K_GEMM, s);
    k_scale_matrix<<<dim3(64, 1, (unsigned)batch), 256, 0, s>>>(C, ldc, sc, (int)m, (int)n, beta);
    return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
  }
  stats_work(K_GEMM, 2.0 * (double)m * (double)n * (double)k * (double)batch);
  if (!transA && !transB && m * n <= 65536 && k <= 1024 && batch <= 65535) {
    LaunchScope ls(K_GEMM, s);
    k_gemm_tiny<<<dim3((unsigned)cdiv(m * n, 256), (unsigned)batch), 256, 0, s>>>((int)m, (int)n, (int)k, alpha, A, lda,
                                                                                  sa, B, ldb, sb, beta, C, ldc, sc);
    return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
  }
  const int64_t target = 2 * num_sms();
  auto tiles = [&](int64_t b) { return cdiv(m, b) * cdiv(n, b) * batch; };
  int bsz = 64;
  if (tiles(64) < target) bsz = 32;
  if (bsz == 32 && tiles(32) < target) bsz = 16;
  int splits = 1;
  const int64_t t = tiles(bsz);
  if (t < target && k >= 256) {
    splits = (int)std::min<int64_t>(cdiv(target, t), k / 128);
    if (splits < 1) splits = 1;
  }
  if (bsz == 64) return launch_gemm<64, 64>(s, transA, transB, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc, batch, splits);
  if (bsz == 32) return launch_gemm<32, 32>(s, transA, transB, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc, batch, splits);
  return launch_gemm<16, 16>(s, transA, transB, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc, batch, splits);
}

size_t qr_f64_scratch(int64_t m, int64_t n) {
  const int64_t nref = m < n ? m : n;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(sizeof(double) * m * (nref > 0 ? nref : 1)) + al(sizeof(double) * (nref + 1)) +
         al(sizeof(unsigned) * (nref + 1));
}

size_t qr_scratch_bound(int64_t max_elems, int64_t max_n) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(sizeof(double) * (max_elems > 0 ? max_elems : 1)) + al(sizeof(double) * (max_n + 1)) +
         al(sizeof(unsigned) * (max_n + 1));
}

int qr_f64(cudaStream_t s, double *A, int64_t m, int64_t n, int64_t lda, double *Rout, int64_t ldr, void *scratch) {
  if (m <= 0 || n <= 0) return TNR_OK;
  const int64_t nref = m < n ? m : n;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  char *p = static_cast<char *>(scratch);
  QrArgs a;
  a.A = A;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.R = Rout;
  a.ldr = ldr;
  a.V = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * m * nref);
  a.tau = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * (nref + 1));
  a.flags = reinterpret_cast<unsigned *>(p);
  a.status = status_ptr();
  TNR_CK(cudaMemsetAsync(a.flags, 0, sizeof(unsigned) * (nref + 1), s));
  int64_t P = std::min<int64_t>(n, num_sms());
  const size_t smem = sizeof(double) * (cdiv(n, P) * m + m);
  if (smem > 200 * 1024) return TNR_EINVAL;  // columns do not fit the shared-memory layout
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  TNR_TRY(ensure_dynamic_smem((const void *)k_qr_coop, smem));
  TNR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_coop, 32, smem));
  if (per_sm < 1) return TNR_ECUDA;
  void *args[] = {&a};
  {
    // dgeqrf + dorgqr operation counts for an m x n matrix with p = min(m, n) reflectors
    const double M = (double)m, N = (double)n, Pq = (double)nref;
    const double fact = m >= n ? 2 * M * N * N - 2 * N * N * N / 3 : 2 * N * M * M - 2 * M * M * M / 3;
    const double org = 2 * M * Pq * Pq - 2 * Pq * Pq * Pq / 3;
    stats_work(K_QR, fact + org);
  }
  LaunchScope ls(K_QR, s);
  TNR_CK(cudaLaunchCooperativeKernel((void *)k_qr_coop, dim3((unsigned)P), dim3(32), args, smem, s));
  return TNR_OK;
}

size_t qrcp_scratch(int64_t m, int64_t n) {
  const int64_t nref = m < n ? m : n;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(sizeof(double) * m * (nref > 0 ? nref : 1)) + al(sizeof(double) * (nref + 1)) +
         al(sizeof(unsigned long long) * (nref + 1)) + al(sizeof(unsigned) * (nref + 2)) +
         al(sizeof(unsigned) * (nref + 1)) + al(sizeof(double)) + al(sizeof(int64_t));
}

size_t qrcp_scratch_bound(int64_t max_elems, int64_t max_n) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(sizeof(double) * (max_elems > 0 ? max_elems : 1)) + al(sizeof(double) * (max_n + 1)) +
         al(sizeof(unsigned long long) * (max_n + 1)) + al(sizeof(unsigned) * (max_n + 2)) +
         al(sizeof(unsigned) * (max_n + 1)) + al(sizeof(double)) + al(sizeof(int64_t));
}

int qrcp_f64(cudaStream_t s, double *A, int64_t m, int64_t n, int64_t lda, double *Rout, int64_t ldr, double cut_rel,
             void *scratch, int64_t *r_dev, bool *used) {
  *used = false;
  if (m <= 0 || n <= 0) return TNR_OK;
  const int64_t nref = m < n ? m : n;
  int64_t P = std::min<int64_t>(n, num_sms());
  const int64_t nc = cdiv(n, P);
  const size_t smem = sizeof(double) * (nc * m + m + nc) + sizeof(int) * nc;
  if (smem > 200 * 1024 || n >= 0xFFFFF) return TNR_OK;  // caller falls back to the unpivoted kernel
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  char *p = static_cast<char *>(scratch);
  QrcpArgs a;
  a.A = A;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.R = Rout;
  a.ldr = ldr;
  a.V = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * m * nref);
  a.tau = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * (nref + 1));
  a.best = reinterpret_cast<unsigned long long *>(p);
  char *zero_begin = p;
  p += al(sizeof(unsigned long long) * (nref + 1));
  a.cnt = reinterpret_cast<unsigned *>(p);
  p += al(sizeof(unsigned) * (nref + 2));
  a.flags = reinterpret_cast<unsigned *>(p);
  p += al(sizeof(unsigned) * (nref + 1));
  a.fro2 = reinterpret_cast<double *>(p);
  p += al(sizeof(double));
  char *zero_end = p;
  a.r_out = r_dev;
  a.cut_rel = cut_rel;
  a.status = status_ptr();
  TNR_CK(cudaMemsetAsync(zero_begin, 0, zero_end - zero_begin, s));
  TNR_TRY(ensure_dynamic_smem((const void *)k_qrcp, smem));
  int per_sm = 0;
  TNR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qrcp, 32, smem));
  if (per_sm < 1) return TNR_OK;
  void *args[] = {&a};
  LaunchScope ls(K_QR, s);
  TNR_CK(cudaLaunchCooperativeKernel((void *)k_qrcp, dim3((unsigned)P), dim3(32), args, smem, s));
  *used = true;
  return TNR_OK;
}

bool qr_small_fits(int64_t m, int64_t n) {
  const int64_t nref = m < n ? m : n;
  const size_t smem = sizeof(double) * (m * n + 2 * n + nref + m) + sizeof(int) * n;
  return smem <= 200 * 1024;
}

int qr_small_f64(cudaStream_t s, const double *src, int64_t lds, int64_t m, int64_t n, bool trans_src, bool pivot,
                 double cut_rel, double *Q, int64_t ldq, bool trans_q, double *R, int64_t ldr, bool trans_r,
                 int64_t *r_dev) {
  if (m <= 0 || n <= 0) return TNR_OK;
  if (!qr_small_fits(m, n)) return TNR_EINVAL;
  const int64_t nref = m < n ? m : n;
  const size_t smem = sizeof(double) * (m * n + n + nref) + sizeof(int) * n;
  QrSmallArgs a;
  a.src = src;
  a.lds = lds;
  a.m = m;
  a.n = n;
  a.trans_src = trans_src;
  a.pivot = pivot;
  a.trans_q = trans_q;
  a.trans_r = trans_r;
  a.cut_rel = cut_rel;
  a.Q = Q;
  a.ldq = ldq;
  a.R = R;
  a.ldr = ldr;
  a.r_out = r_dev;
  {
    const double M = (double)m, N = (double)n, P = (double)nref;
    // pivoted calls stop early: their work is recorded by the caller once the rank is known
    if (!pivot) stats_work(K_QR_SMALL, 2 * M * N * P - (M + N) * P * P + 2 * P * P * P / 3 + 2 * M * P * P - 2 * P * P * P / 3);
  }
  if (m <= 64) {  // short columns: one thread per column
    const size_t sm2 = sizeof(double) * (m * n + 2 * n + nref + m) + sizeof(int) * n;
    TNR_TRY(ensure_dynamic_smem((const void *)k_qr_small_tpc, sm2));
    LaunchScope ls(pivot ? K_QR_PIV : K_QR_SMALL, s);
    k_qr_small_tpc<<<1, kSmallThreads, sm2, s>>>(a);
    return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
  }
  TNR_TRY(ensure_dynamic_smem((const void *)k_qr_small, smem));
  LaunchScope ls(pivot ? K_QR_PIV : K_QR_SMALL, s);
  k_qr_small<<<1, kSmallThreads, smem, s>>>(a);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// CTAs of the K x K Jacobi's cluster, and whether cluster launches work in this process
// (-1 unknown, 0 refused, 1 working).
constexpr int kJacCluster = 8;
static std::atomic<int> g_jac_cluster{-1};

// Doubles of the K x K Jacobi's working set: G, V and the mixed-precision work area.
static int64_t jacobi_elems(int64_t n) { return 2 * n * n + jacobi_mixed_work(n) + jacobi_refine_work(n); }

size_t jacobi_scratch(int64_t n) {
  if (jacobi_elems(n) * (int64_t)sizeof(double) <= 160 * 1024) return 0;
  return ((size_t)jacobi_elems(n) * sizeof(double) + 255) & ~size_t(255);
}

int jacobi_svd_f64(cudaStream_t s, double *G, int64_t n, int64_t ldg, double *S, double *V, int64_t ldv,
                   void *scratch) {
  if (n <= 0) return TNR_OK;
  if (n > 1024) return TNR_EINVAL;
  double *Gw = nullptr, *Vw = nullptr;
  size_t smem = (size_t)jacobi_elems(n) * sizeof(double);
  if (smem > 160 * 1024) {
    Gw = static_cast<double *>(scratch);
    Vw = Gw + n * n;  // the mixed sweeps' work area follows V
    smem = 0;
  }
  TNR_TRY(ensure_dynamic_smem((const void *)k_jacobi, smem));
  const int ppw = jacobi_pairs_per_warp((int)n, kJacThreads / 32);
  // at least eight warps: the sweeps use those their pairs need, the refinement's FP64 products all
  // (one warp per SM sub-partition leaves the FMA latency exposed); up to 32 columns, one warp per
  // column pair of the FP32 sweeps
  int64_t want = std::max<int64_t>(8, ((n + 1) / 2 + ppw - 1) / ppw);
  if (n <= 32) want = std::max<int64_t>(want, (n + 1) / 2);
  const int warps = (int)std::min<int64_t>(kJacThreads / 32, want);
  LaunchScope ls(K_SVD, s);
  // working set in shared memory: a cluster of kJacCluster CTAs shares the refinement's products
  // (one GPU; distributed shared memory), unless cluster launches were refused before
  if (Gw == nullptr && n <= 32 && g_jac_cluster.load() != 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)kJacCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)kJacCluster);
    cfg.blockDim = dim3((unsigned)(32 * warps));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_jacobi, G, (int)n, (int)ldg, S, V, (int)ldv, Gw, Vw, status_ptr());
    if (e == cudaSuccess) {
      g_jac_cluster.store(1);
      return TNR_OK;
    }
    (void)cudaGetLastError();  // refused: one CTA from now on
    g_jac_cluster.store(0);
  }
  k_jacobi<<<1, 32 * warps, smem, s>>>(G, (int)n, (int)ldg, S, V, (int)ldv, Gw, Vw, status_ptr());
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

int copy_matrix_f64(cudaStream_t s, const double *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                    bool transpose) {
  if (m <= 0 || n <= 0) return TNR_OK;
  LaunchScope ls(K_MISC, s);
  k_copy<<<grid_for(m * n), 256, 0, s>>>(src, lds, dst, ldd, (int)m, (int)n, transpose ? 1 : 0);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

int scale_columns_f64(cudaStream_t s, double *A, int64_t lda, int64_t m, int64_t n, const double *scale) {
  if (m <= 0 || n <= 0) return TNR_OK;
  LaunchScope ls(K_MISC, s);
  k_scale_cols<<<grid_for(m * n), 256, 0, s>>>(A, lda, (int)m, (int)n, scale);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

}  // namespace tnr
