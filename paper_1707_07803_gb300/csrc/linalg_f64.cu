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
#include <cstdio>

#include "tnr_internal.cuh"

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

__global__ void k_scale_matrix(double *C, int64_t ldc, int64_t sc, int64_t m, int64_t n, double beta) {
  const int64_t b = blockIdx.z;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n; idx += (int64_t)gridDim.x * blockDim.x) {
    double *c = C + b * sc + (idx % m) + ldc * (idx / m);
    *c = beta == 0.0 ? 0.0 : beta * *c;
  }
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
    k_scale_matrix<<<dim3(64, 1, (unsigned)batch), 256, 0, s>>>(C, ldc, sc, m, n, beta);
  }
  LaunchScope ls(K_GEMM, s);
#define TNR_G(TA_, TB_) \
  k_gemm<BM, BN, TA_, TB_><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc, splits, kchunk)
  if (!ta && !tb) TNR_G(false, false);
  else if (ta && !tb) TNR_G(true, false);
  else if (!ta && tb) TNR_G(false, true);
  else TNR_G(true, true);
#undef TNR_G
  return check_cuda(cudaGetLastError());
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

// ------------------------------------------------------------------------------------------
// Householder QR, columns distributed cyclically over P CTAs (cooperative launch, so all CTAs
// are resident). Reflector j (LAPACK dlarfg convention: beta = -sign(alpha) ||x||,
// tau = (beta - alpha) / beta, v = x / (alpha - beta), v_j = 1) is computed by the owner of
// column j, written to V[:, j] and published with a release store to flags[j]; every CTA
// applies it to its own columns after an acquire load. The owner of column j+1 applies
// reflector j to column j+1 first and publishes reflector j+1 before updating its other
// columns (one-column lookahead), so the critical path per column is one flag hop plus one
// column update. Waits are bounded (kSpinCap polls); on timeout the kernel records
// TNR_ETIMEOUT and returns.
// ------------------------------------------------------------------------------------------
constexpr int kQrThreads = 256;

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

__device__ void qr_make_reflector(const QrArgs &a, int64_t j, double *red) {
  double *col = a.A + a.lda * j;
  double sig = 0.0;
  for (int64_t i = j + 1 + threadIdx.x; i < a.m; i += kQrThreads) sig = fma(col[i], col[i], sig);
  sig = block_sum<kQrThreads>(sig, red);
  const double alpha = col[j];
  double tau = 0.0, beta = alpha, scal = 0.0;
  if (sig > 0.0) {
    beta = -copysign(sqrt(fma(alpha, alpha, sig)), alpha);
    tau = (beta - alpha) / beta;
    scal = 1.0 / (alpha - beta);
  }
  double *v = a.V + a.m * j;
  for (int64_t i = j + 1 + threadIdx.x; i < a.m; i += kQrThreads) v[i] = col[i] * scal;
  if (threadIdx.x == 0) {
    v[j] = 1.0;
    col[j] = beta;
    a.tau[j] = tau;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(a.flags + j, 1u);
  }
}

// Apply H_j = I - tau v v^T (v from vs, rows j..m-1) to column l of A.
__device__ __forceinline__ void qr_apply(const QrArgs &a, const double *vs, double tau, int64_t j, int64_t l,
                                         double *red) {
  double *col = a.A + a.lda * l;
  double w = 0.0;
  for (int64_t i = j + threadIdx.x; i < a.m; i += kQrThreads) w = fma(vs[i - j], col[i], w);
  w = block_sum<kQrThreads>(w, red) * tau;
  for (int64_t i = j + threadIdx.x; i < a.m; i += kQrThreads) col[i] = fma(-w, vs[i - j], col[i]);
  __syncthreads();
}

__global__ void __launch_bounds__(kQrThreads) k_qr_coop(QrArgs a) {
  extern __shared__ double vs[];  // m doubles: the current reflector
  __shared__ double red[kQrThreads / 32];
  __shared__ int s_abort;
  const int64_t P = gridDim.x, c = blockIdx.x;
  const int64_t nref = a.m < a.n ? a.m : a.n;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  if (c == 0 && nref > 0) qr_make_reflector(a, 0, red);
  for (int64_t j = 0; j < nref; ++j) {
    // my first owned column > j
    int64_t l0 = j + 1 + ((c - (j + 1) % P) + P) % P;
    if (l0 >= a.n) break;  // nothing left for this CTA (owned columns only grow)
    if (threadIdx.x == 0) {
      long long spins = 0;
      while (ld_acquire(a.flags + j) == 0u) {
        if (++spins > kSpinCap) {
          set_status(a.status, TNR_ETIMEOUT);
          s_abort = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (s_abort) return;
    for (int64_t i = j + threadIdx.x; i < a.m; i += kQrThreads) vs[i - j] = __ldcg(a.V + a.m * j + i);
    const double tau = __ldcg(a.tau + j);
    __syncthreads();
    if (tau != 0.0) {
      for (int64_t l = l0; l < a.n; l += P) {
        qr_apply(a, vs, tau, j, l, red);
        if (l == j + 1 && l < nref) qr_make_reflector(a, l, red);
      }
    } else if (l0 == j + 1 && l0 < nref) {
      qr_make_reflector(a, l0, red);
    }
    __syncthreads();
  }
  // R: column l of the upper trapezoid (rows 0..min(l, nref-1)), zeros below.
  for (int64_t l = c; l < a.n; l += P) {
    const double *col = a.A + a.lda * l;
    for (int64_t i = threadIdx.x; i < nref; i += kQrThreads) a.R[i + a.ldr * l] = i <= l ? col[i] : 0.0;
  }
  __syncthreads();
  // Explicit Q, column c' = H_0 ... H_{c'} e_{c'} for my columns c' < nref. All reflectors
  // j <= c' were observed above (owner of c' waited for every j < c' and made c' itself).
  for (int64_t l = c; l < nref; l += P) {
    double *q = a.A + a.lda * l;
    for (int64_t i = threadIdx.x; i < a.m; i += kQrThreads) q[i] = (i == l) ? 1.0 : 0.0;
    __syncthreads();
    for (int64_t j = l; j >= 0; --j) {
      const double tau = __ldcg(a.tau + j);
      if (tau == 0.0) continue;
      const double *v = a.V + a.m * j;
      double w = 0.0;
      for (int64_t i = j + threadIdx.x; i < a.m; i += kQrThreads) w = fma(__ldcg(v + i), q[i], w);
      w = block_sum<kQrThreads>(w, red) * tau;
      for (int64_t i = j + threadIdx.x; i < a.m; i += kQrThreads) q[i] = fma(-w, __ldcg(v + i), q[i]);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------------------
// One-sided Jacobi SVD of an n x n matrix in one CTA (Hestenes): rotate column pairs of G,
// accumulating V, until every pair is orthogonal to |g_p^T g_q| <= tol ||g_p|| ||g_q||.
// Pairs follow a round-robin tournament, so each round's pairs are disjoint and are
// processed by different warps. Results sorted by descending singular value.
// ------------------------------------------------------------------------------------------
constexpr int kJacThreads = 512;

__global__ void __launch_bounds__(kJacThreads) k_jacobi(double *G, int64_t n, int64_t ldg, double *S, double *V,
                                                        int64_t ldv, double *Gw, double *Vw, int *status) {
  extern __shared__ double sm[];
  __shared__ int s_rot;
  __shared__ double s_norm[1024];
  const bool in_smem = Gw == nullptr;
  double *g = in_smem ? sm : Gw;        // working copy, ld n
  double *v = in_smem ? sm + n * n : Vw;  // working V, ld n
  for (int64_t idx = threadIdx.x; idx < n * n; idx += kJacThreads) {
    const int64_t i = idx % n, j = idx / n;
    g[idx] = G[i + ldg * j];
    v[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = kJacThreads / 32;
  const int64_t np = (n + 1) & ~int64_t(1);  // even number of players
  const double tol = DBL_EPSILON * (double)(n > 8 ? n : 8);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int64_t round = 0; round < np - 1; ++round) {
      for (int64_t pr = warp; pr < np / 2; pr += nw) {
        int64_t p, q;
        if (pr == 0) {
          p = round;
          q = np - 1;
        } else {
          p = (round + pr) % (np - 1);
          q = (round - pr + (np - 1)) % (np - 1);
        }
        if (p >= n || q >= n) continue;
        if (p > q) {
          int64_t t = p;
          p = q;
          q = t;
        }
        double *gp = g + n * p, *gq = g + n * q;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int64_t i = lane; i < n; i += 32) {
          const double x = gp[i], y = gq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == 0.0 || al == 0.0 || be == 0.0) continue;
        if (fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        const double cs = 1.0 / sqrt(fma(t, t, 1.0)), sn = cs * t;
        for (int64_t i = lane; i < n; i += 32) {
          const double x = gp[i], y = gq[i];
          gp[i] = cs * x - sn * y;
          gq[i] = sn * x + cs * y;
        }
        double *vp = v + n * p, *vq = v + n * q;
        for (int64_t i = lane; i < n; i += 32) {
          const double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (!s_rot) break;
  }
  // column norms
  for (int64_t j = warp; j < n; j += nw) {
    double s = 0.0;
    for (int64_t i = lane; i < n; i += 32) s = fma(g[i + n * j], g[i + n * j], s);
    s = warp_sum(s);
    if (lane == 0) s_norm[j] = sqrt(s);
  }
  __syncthreads();
  // rank of each column by descending norm (stable), then scatter.
  for (int64_t j = warp; j < n; j += nw) {
    const double sj = s_norm[j];
    int64_t rank = 0;
    for (int64_t i = lane; i < n; i += 32) {
      const double si = s_norm[i];
      rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    for (int64_t i = lane; i < n; i += 32) {
      G[i + ldg * rank] = g[i + n * j] * inv;
      V[i + ldv * rank] = v[i + n * j];
    }
    if (lane == 0) S[rank] = sj;
  }
}

__global__ void k_copy(const double *__restrict__ src, int64_t lds, double *__restrict__ dst, int64_t ldd, int64_t m,
                       int64_t n, int transpose) {
  // dst (m x n) = src (m x n) or src^T (src is n x m when transposing)
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
    dst[i + ldd * j] = transpose ? src[j + lds * i] : src[i + lds * j];
  }
}

__global__ void k_scale_cols(double *A, int64_t lda, int64_t m, int64_t n, const double *scale) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
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
    k_scale_matrix<<<dim3(64, 1, (unsigned)batch), 256, 0, s>>>(C, ldc, sc, m, n, beta);
    return check_cuda(cudaGetLastError());
  }
  stats_work(K_GEMM, 2.0 * (double)m * (double)n * (double)k * (double)batch);
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
  const size_t smem = sizeof(double) * m;
  if (smem > 200 * 1024) return TNR_EINVAL;  // m > 25600 rows: outside the supported sizes
  int64_t P = n;
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  if (smem > 48 * 1024) TNR_CK(cudaFuncSetAttribute(k_qr_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TNR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_coop, kQrThreads, smem));
  const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? 1 : 0);
  if (P > cap) P = cap;
  if (P < 1) return TNR_ECUDA;
  void *args[] = {&a};
  {
    // dgeqrf + dorgqr operation counts for an m x n matrix with p = min(m, n) reflectors
    const double M = (double)m, N = (double)n, Pq = (double)nref;
    const double fact = m >= n ? 2 * M * N * N - 2 * N * N * N / 3 : 2 * N * M * M - 2 * M * M * M / 3;
    const double org = 2 * M * Pq * Pq - 2 * Pq * Pq * Pq / 3;
    stats_work(K_QR, fact + org);
  }
  LaunchScope ls(K_QR, s);
  TNR_CK(cudaLaunchCooperativeKernel((void *)k_qr_coop, dim3((unsigned)P), dim3(kQrThreads), args, smem, s));
  return TNR_OK;
}

size_t jacobi_scratch(int64_t n) {
  if (2 * n * n * sizeof(double) <= 160 * 1024) return 0;
  return 2 * (((size_t)n * n * sizeof(double) + 255) & ~size_t(255));
}

int jacobi_svd_f64(cudaStream_t s, double *G, int64_t n, int64_t ldg, double *S, double *V, int64_t ldv,
                   void *scratch) {
  if (n <= 0) return TNR_OK;
  if (n > 1024) return TNR_EINVAL;
  double *Gw = nullptr, *Vw = nullptr;
  size_t smem = 2 * n * n * sizeof(double);
  if (smem > 160 * 1024) {
    Gw = static_cast<double *>(scratch);
    Vw = Gw + (((size_t)n * n * sizeof(double) + 255) & ~size_t(255)) / sizeof(double);
    smem = 0;
  }
  if (smem > 48 * 1024) TNR_CK(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LaunchScope ls(K_SVD, s);
  k_jacobi<<<1, kJacThreads, smem, s>>>(G, n, ldg, S, V, ldv, Gw, Vw, status_ptr());
  return check_cuda(cudaGetLastError());
}

int copy_matrix_f64(cudaStream_t s, const double *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                    bool transpose) {
  if (m <= 0 || n <= 0) return TNR_OK;
  LaunchScope ls(K_MISC, s);
  k_copy<<<grid_for(m * n), 256, 0, s>>>(src, lds, dst, ldd, m, n, transpose ? 1 : 0);
  return check_cuda(cudaGetLastError());
}

int scale_columns_f64(cudaStream_t s, double *A, int64_t lda, int64_t m, int64_t n, const double *scale) {
  if (m <= 0 || n <= 0) return TNR_OK;
  LaunchScope ls(K_MISC, s);
  k_scale_cols<<<grid_for(m * n), 256, 0, s>>>(A, lda, m, n, scale);
  return check_cuda(cudaGetLastError());
}

}  // namespace tnr
