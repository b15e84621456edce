// TNrSVD of a sparse matrix in the block form of Alg. 4.1.
//
// Alg. 4.1 turns a sparse matrix into a sum of R rank-1 MPOs, one per nonzero I_1 x J_1 block
// (Eq. (4.1)), so the MPO has rank R at every bond (Lemma 4.2) and MPO-times-MPO products
// (Section 5.2) would multiply ranks by R (5.5 million for a 2^20 banded matrix). The same
// operator is applied here straight from the block form: block t adds X_t times rows
// q_t J_1 .. q_t J_1 + J_1 - 1 of the right-hand side to rows p_t I_1 .. of the result (A Q), and
// X_t^T times rows p_t I_1 .. to rows q_t J_1 .. (A^T Q), where p_t, q_t are the block row and
// column numbers in the mixed radix of the digits (Eq. (2.1)). Omega (Lemma 5.1, over the merged
// column dims of Section 6.3) is expanded to its dense (prod J) x K matrix, and Alg. 5.4 / 5.1
// run on dense tall matrices: Y = A Omega, Q = qr(Y), q times { Q = qr(A^T Q), Q = qr(A Q) },
// Z = A^T Q (= B^T), Z = Qz Rz, SVD Rz^T = W S Zr^T, U = Q W, V = Qz Zr. Without truncation this
// is TNrSVD in exact arithmetic (the MPO products and roundings are exact).
//
// GB300 mapping: the blocks' nonzeros are gathered once into compact row and column lists (the
// 4 x 4 blocks of a banded matrix hold ~1.5 nonzeros each), the tall matrices are row-major, and a
// product is one warp per output row with lanes over the K columns: per nonzero one coalesced
// row load and one FMA per lane, sums in index order (deterministic). The tall-skinny QRs are
// CholeskyQR2 (a pass whose Cholesky breaks down is redone with the shift of shifted CholeskyQR3,
// Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020): a symmetric FP64 Gram pass and a
// row-parallel triangular solve per factor instead of a Householder chain over 2^20 rows.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cholqr.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

int grid_n(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), 152 * 32));
}

// p_t, q_t of every block from its digits (i_2, j_2, i_3, j_3, ...), checking block order
__global__ void k_block_pq(const uint8_t *__restrict__ digits, int64_t R, int dm1, const int64_t *__restrict__ I,
                           const int64_t *__restrict__ J, int *p, int *q, int *status) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < R; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t pp = 0, qq = 0, sp = 1, sq = 1;
    for (int k = 0; k < dm1; ++k) {
      const int64_t di = digits[t * 2 * dm1 + 2 * k], dj = digits[t * 2 * dm1 + 2 * k + 1];
      if (di >= I[k + 1] || dj >= J[k + 1]) set_status(status, TNR_ERANGE);
      pp += di * sp;
      qq += dj * sq;
      sp *= I[k + 1];
      sq *= J[k + 1];
    }
    p[t] = (int)pp;
    q[t] = (int)qq;
  }
}

// exclusive scan of n ints into out[0..n] in three launches: per-tile scans (kScanTile ints per CTA)
// with tile totals, a one-CTA scan of the totals, and the tile offsets added back
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int *__restrict__ in, int64_t n, int *out, int *tot) {
  __shared__ int warp_sums[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer], s = 0;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    v[u] = base + u < n ? in[base + u] : 0;
    s += v[u];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int run = incl - s + (warp > 0 ? warp_sums[warp - 1] : 0);
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    if (base + u < n) out[base + u] = run;
    run += v[u];
  }
  if (threadIdx.x == kScanThreads - 1) tot[blockIdx.x] = warp_sums[31];
}

__global__ void __launch_bounds__(1024) k_scan_small(int *tot, int64_t nt, int *total_out) {
  __shared__ int part[1024];
  const int64_t per = cdiv(nt, 1024);
  const int64_t b = threadIdx.x * per, e = (b + per < nt) ? b + per : nt;
  int s = 0;
  for (int64_t i = b; i < e; ++i) s += tot[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < 1024; ++i) {
      const int v = part[i];
      part[i] = acc;
      acc += v;
    }
    *total_out = acc;
  }
  __syncthreads();
  int acc = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) {
    const int v = tot[i];
    tot[i] = acc;
    acc += v;
  }
}

__global__ void k_scan_add(int *out, int64_t n, const int *__restrict__ tot) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    out[x] += tot[x / kScanTile];
}

// dense Omega (ncols x K, row-major): row j = j1 + J1 (j2 + J2 (...)) over the merged dims Jm
__global__ void k_omega_dense(const double *__restrict__ draws, int dmm, const int64_t *__restrict__ Jm, int64_t K,
                              int64_t ncols, double *O) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ncols * K;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = x % K, row = x / K;
    int64_t rem = row / Jm[0];
    const int64_t j1 = row % Jm[0];
    double v = draws[j1 + Jm[0] * c];
    int64_t pos = Jm[0] * K;
    for (int k = 1; k < dmm; ++k) {
      v *= draws[pos + rem % Jm[k]];
      pos += Jm[k];
      rem /= Jm[k];
    }
    O[x] = v;
  }
}

// Nonzeros of the blocks, counted per row (by_col = 0) or per column (by_col = 1). The 4 x 4 blocks
// of Alg. 4.1 hold few nonzeros each (a 2^20 banded matrix: ~1.5 of 16), so the products run over
// compact row and column lists built once from the block form instead of the dense blocks.
__global__ void k_nz_count(const double *__restrict__ X, const int *__restrict__ p, const int *__restrict__ q,
                           int64_t R, int I1, int J1, int by_col, int *cnt) {
  const int64_t bs = (int64_t)I1 * J1;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < R * bs; x += (int64_t)gridDim.x * blockDim.x) {
    if (X[x] == 0.0) continue;
    const int64_t t = x / bs, e = x % bs, i = e % I1, j = e / I1;
    atomicAdd(&cnt[by_col ? (int64_t)q[t] * J1 + j : (int64_t)p[t] * I1 + i], 1);
  }
}

__global__ void k_nz_fill(const double *__restrict__ X, const int *__restrict__ p, const int *__restrict__ q, int64_t R,
                          int I1, int J1, int by_col, const int *__restrict__ ptr, int *cursor, int *idx, double *val) {
  const int64_t bs = (int64_t)I1 * J1;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < R * bs; x += (int64_t)gridDim.x * blockDim.x) {
    const double v = X[x];
    if (v == 0.0) continue;
    const int64_t t = x / bs, e = x % bs, i = e % I1, j = e / I1;
    const int64_t row = (int64_t)p[t] * I1 + i, col = (int64_t)q[t] * J1 + j;
    const int64_t key = by_col ? col : row;
    const int64_t at = ptr[key] + atomicAdd(&cursor[key], 1);
    idx[at] = (int)(by_col ? row : col);
    val[at] = v;
  }
}

// each list in increasing index order (deterministic summation order)
__global__ void k_sort_lists(const int *__restrict__ ptr, int64_t n, int *idx, double *val) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int b = ptr[r], e = ptr[r + 1];
    for (int i = b + 1; i < e; ++i) {
      const int ki = idx[i];
      const double vi = val[i];
      int j = i - 1;
      while (j >= b && idx[j] > ki) {
        idx[j + 1] = idx[j];
        val[j + 1] = val[j];
        --j;
      }
      idx[j + 1] = ki;
      val[j + 1] = vi;
    }
  }
}

// Y (n x K, row-major: (r, c) at c + K r) = A Q, with A given by its compact row lists (ptr, idx,
// val) and Q row-major: one warp per output row, lanes over the columns (chunks of 32), so every
// nonzero costs one coalesced load of a row of Q and one FMA per lane. T is the multiply-add type.
template <typename T>
__global__ void __launch_bounds__(256) k_spmm_rows(const int *__restrict__ ptr, const int *__restrict__ idx,
                                                   const double *__restrict__ val, const double *__restrict__ Qd,
                                                   int64_t n, int64_t K, double *Y) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int b = ptr[r], e = ptr[r + 1];
    for (int64_t c0 = 0; c0 < K; c0 += 32) {
      const int64_t c = c0 + lane;
      T acc = 0;
      if (c < K)
        for (int u = b; u < e; ++u) acc = fma((T)val[u], (T)Qd[(int64_t)idx[u] * K + c], acc);
      if (c < K) Y[r * K + c] = (double)acc;
    }
  }
}

// Cholesky G = R^T R (K x K, upper R) in one CTA, G in shared memory; shift s added to the
// diagonal first. Writes R (ld K) with zeros below; status ENONFINITE on a non-positive pivot.
__global__ void __launch_bounds__(256) k_chol(const double *__restrict__ G, int64_t K, double shift, double *Rout,
                                              double *rdiag, int *status) {
  extern __shared__ double a[];
  for (int64_t x = threadIdx.x; x < K * K; x += blockDim.x) a[x] = G[x] + ((x % K == x / K) ? shift : 0.0);
  __syncthreads();
  __shared__ double s_inv;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int64_t j = 0; j < K; ++j) {
    if (threadIdx.x == 0) {
      const double dj = a[j + K * j];
      if (!(dj > 0.0) || !isfinite(dj)) {
        s_bad = 1;
        s_inv = 0.0;
      } else {
        const double r = sqrt(dj);
        a[j + K * j] = r;
        s_inv = 1.0 / r;
        rdiag[j] = s_inv;
      }
    }
    __syncthreads();
    if (s_bad) break;
    // row j of R: R(j, l) = a(j, l) / R(j, j) for l > j (upper part holds the working matrix)
    for (int64_t l = j + 1 + threadIdx.x; l < K; l += blockDim.x) a[j + K * l] *= s_inv;
    __syncthreads();
    // trailing update a(i, l) -= R(j, i) R(j, l), i <= l
    for (int64_t x = threadIdx.x; x < (K - j - 1) * (K - j - 1); x += blockDim.x) {
      const int64_t i = j + 1 + x % (K - j - 1), l = j + 1 + x / (K - j - 1);
      if (i <= l) a[i + K * l] = fma(-a[j + K * i], a[j + K * l], a[i + K * l]);
    }
    __syncthreads();
  }
  if (s_bad && threadIdx.x == 0) set_status(status, TNR_ENONFINITE);
  for (int64_t x = threadIdx.x; x < K * K; x += blockDim.x) Rout[x] = (x % K <= x / K) ? a[x] : 0.0;
}

// Y (n x K, row-major) <- Y R^{-1}, R upper (K x K, column-major), rdiag = 1 / diag(R): thread per
// row, forward substitution (reciprocals formed once: FP64 division is a long instruction sequence)
__global__ void k_trsm_rm(double *Y, int64_t n, int64_t K, const double *__restrict__ R, const double *__restrict__ rdiag) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double *y = Y + r * K;
    for (int64_t j = 0; j < K; ++j) {
      double acc = y[j];
      for (int64_t l = 0; l < j; ++l) acc = fma(-y[l], R[l + K * j], acc);
      y[j] = acc * rdiag[j];
    }
  }
}

struct SBufs {
  int *p, *q, *rcnt, *rptr, *ridx, *ccnt, *cptr, *cidx, *tiles;
  double *rval, *cval;
  double *draws, *O, *Y, *Q, *Z, *G, *R1, *Rt, *Racc, *Sv, *Vk, *rdiag;
  void *jac;
};

int gram(cudaStream_t s, const double *Y, int64_t n, int64_t K, double *G) {
  TNR_CK(cudaMemsetAsync(G, 0, sizeof(double) * K * K, s));
  const size_t smem = sizeof(double) * kGramRows * K;
  TNR_TRY(ensure_dynamic_smem((const void *)k_gram_rm, smem));
  LaunchScope ls(K_GEMM, s);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(cdiv(n, kGramRows), 152 * 4));
  k_gram_rm<<<(unsigned)blocks, kGramThreads, smem, s>>>(Y, n, K, G);
  stats_work(K_GEMM, (double)n * K * (K + 1));
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// Q R of the tall row-major Y (n x K) in place: CholeskyQR2 (two passes of Gram -> Cholesky ->
// Y R^{-1}); when a Cholesky breaks down (cond(Y) beyond ~1e8) that pass is redone with the shift
// of shifted CholeskyQR3 (Fukaya et al. 2020: s = 11 (n K + K (K + 1)) u ||Y||_F^2) and one more
// plain pass follows. want_r: the product of the triangular factors goes to b.Racc.
int chol_qr(cudaStream_t s, double *Y, int64_t n, int64_t K, SBufs &b, bool want_r) {
  int passes = 2;
  bool shifted = false;
  for (int pass = 0; pass < passes; ++pass) {
    TNR_TRY(gram(s, Y, n, K, b.G));
    double shift = 0.0;
    if (shifted) {
      std::vector<double> g(K * K);
      TNR_CK(cudaMemcpyAsync(g.data(), b.G, sizeof(double) * K * K, cudaMemcpyDeviceToHost, s));
      TNR_TRY(read_status(s));
      double tr = 0.0;
      for (int64_t i = 0; i < K; ++i) tr += g[i + K * i];
      shift = 11.0 * ((double)n * K + (double)K * (K + 1)) * 1.1102230246251565e-16 * tr;
    }
    {
      LaunchScope ls(K_QR, s);
      TNR_TRY(ensure_dynamic_smem((const void *)k_chol, sizeof(double) * K * K));
      k_chol<<<1, 256, sizeof(double) * K * K, s>>>(b.G, K, shift, b.R1, b.rdiag, status_ptr());
    }
    TNR_CK(cudaGetLastError());
    const int st = read_status(s);
    if (st == TNR_ENONFINITE && !shifted) {  // redo this pass shifted, then one more plain pass
      shifted = true;
      passes += 1;
      --pass;
      continue;
    }
    if (st != TNR_OK) return st;
    shifted = false;
    {
      LaunchScope ls(K_QR, s);
      k_trsm_rm<<<grid_n(n), 256, 0, s>>>(Y, n, K, b.R1, b.rdiag);
      stats_work(K_QR, (double)n * K * K);
    }
    TNR_CK(cudaGetLastError());
    if (want_r) {  // Racc <- R1 Racc
      if (pass == 0) {
        TNR_CK(cudaMemcpyAsync(b.Racc, b.R1, sizeof(double) * K * K, cudaMemcpyDeviceToDevice, s));
      } else {
        TNR_TRY(gemm_f64(s, false, false, K, K, K, 1.0, b.R1, K, 0, b.Racc, K, 0, 0.0, b.Rt, K, 0));
        TNR_CK(cudaMemcpyAsync(b.Racc, b.Rt, sizeof(double) * K * K, cudaMemcpyDeviceToDevice, s));
      }
    }
  }
  return TNR_OK;
}

struct SDims {
  int64_t nrows, ncols, R, K, P, C;
  int I1, J1;
};

// out (n_out x K, row-major) = (A or A^T) in (n_in x K, row-major) over compact lists
// FP64 multiply-adds in both precisions: the double -> float conversions run on the FP64 pipe,
// so an FP32 product of FP64 data costs more issue slots than the FP64 FMA it would replace.
int spmm(cudaStream_t s, const int *ptr, const int *idx, const double *val, int64_t n_out, int64_t n_in, int64_t K,
         const double *in, double *out, int64_t nnz) {
  LaunchScope ls(K_CONTRACT, s);
  const int64_t threads = n_out * 32;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(threads, 256), 152 * 64));
  k_spmm_rows<double><<<grid, 256, 0, s>>>(ptr, idx, val, in, n_out, K, out);
  stats_work(K_CONTRACT, 12.0 * (double)nnz + 4.0 * (double)(n_out + 1) + 8.0 * (double)(n_in + n_out) * K);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

int sparse_dims(int64_t nrows, int64_t ncols, int32_t d, const int64_t *I, const int64_t *J, int32_t k, int32_t p,
                SDims &D, int &m, std::vector<int64_t> &Jm) {
  if (d < 1 || d > TNR_MAX_SITES || !I || !J || k < 1 || p < 0) return TNR_EINVAL;
  double pi = 1, pj = 1;
  for (int i = 0; i < d; ++i) {
    if (I[i] < 1 || J[i] < 1 || I[i] > 256 || J[i] > 256) return TNR_EINVAL;
    pi *= (double)I[i];
    pj *= (double)J[i];
  }
  if (pi != (double)nrows || pj != (double)ncols) return TNR_EINVAL;
  if (nrows > (1LL << 31) || ncols > (1LL << 31)) return TNR_ERANGE;
  D.nrows = nrows;
  D.ncols = ncols;
  D.K = (int64_t)k + p;
  D.I1 = (int)I[0];
  D.J1 = (int)J[0];
  D.P = nrows / I[0];
  D.C = ncols / J[0];
  m = 0;
  pi = pj = 1;
  for (int i = 0; i < d; ++i) {
    pi *= (double)I[i];
    pj *= (double)J[i];
    if (pi >= (double)D.K && pj >= (double)D.K) {
      m = i + 1;
      break;
    }
  }
  if (m == 0) return TNR_EINVAL;
  Jm.assign(1, 1);
  for (int i = 0; i < m; ++i) Jm[0] *= J[i];
  for (int i = m; i < d; ++i) Jm.push_back(J[i]);
  return TNR_OK;
}

void carve_sparse(Arena &ar, const SDims &D, int64_t R, int64_t olen, SBufs &b) {
  const int64_t N = std::max(D.nrows, D.ncols), K = D.K, nzcap = std::max<int64_t>(R * D.I1 * D.J1, 1);
  b.p = ar.take<int>(std::max<int64_t>(R, 1));
  b.q = ar.take<int>(std::max<int64_t>(R, 1));
  b.rcnt = ar.take<int>(D.nrows + 1);
  b.rptr = ar.take<int>(D.nrows + 1);
  b.ccnt = ar.take<int>(D.ncols + 1);
  b.cptr = ar.take<int>(D.ncols + 1);
  b.ridx = ar.take<int>(nzcap);
  b.tiles = ar.take<int>(cdiv(N + 1, kScanTile) + 1);
  b.cidx = ar.take<int>(nzcap);
  b.rval = ar.take<double>(nzcap);
  b.cval = ar.take<double>(nzcap);
  b.draws = ar.take<double>(olen);
  b.O = ar.take<double>(D.ncols * K);
  b.Y = ar.take<double>(N * K);
  b.Q = ar.take<double>(N * K);
  b.Z = ar.take<double>(N * K);
  b.G = ar.take<double>(K * K);
  b.R1 = ar.take<double>(K * K);
  b.Rt = ar.take<double>(K * K);
  b.Racc = ar.take<double>(K * K);
  b.Sv = ar.take<double>(K);
  b.Vk = ar.take<double>(K * K);
  b.rdiag = ar.take<double>(K);
  b.jac = ar.take<char>(std::max<size_t>(jacobi_scratch(K), 256));
}

int64_t omega_len(const std::vector<int64_t> &Jm, int64_t K) {
  int64_t n = Jm[0] * K;
  for (size_t i = 1; i < Jm.size(); ++i) n += Jm[i];
  return n;
}

}  // namespace
}  // namespace tnr

extern "C" int tnr_sparse_solve_workspace(int64_t nrows, int64_t ncols, int64_t R, int32_t d, const int64_t *I,
                                          const int64_t *J, int32_t k, int32_t p, size_t *bytes) {
  using namespace tnr;
  if (!bytes || R < 0) return TNR_EINVAL;
  SDims D;
  int m = 0;
  std::vector<int64_t> Jm;
  TNR_TRY(sparse_dims(nrows, ncols, d, I, J, k, p, D, m, Jm));
  Arena ar;
  SBufs b;
  carve_sparse(ar, D, R, omega_len(Jm, D.K), b);
  *bytes = ar.off + (size_t)2 * 8 * TNR_MAX_SITES + 512;
  return TNR_OK;
}

extern "C" int tnr_sparse_solve(int64_t nrows, int64_t ncols, int64_t R, const double *X, const uint8_t *digits,
                                int32_t d, const int64_t *I, const int64_t *J, int32_t k, int32_t p, int32_t q,
                                uint64_t seed, int32_t precision, double *U, double *S, double *V, void *ws,
                                size_t ws_bytes, void *stream) {
  using namespace tnr;
  if (R < 1 || !X || (d > 1 && !digits) || q < 0 || !U || !S || !V || !ws) return TNR_EINVAL;
  if (precision != TNR_FP64 && precision != TNR_MIXED) return TNR_EINVAL;
  SDims D;
  int m = 0;
  std::vector<int64_t> Jm;
  TNR_TRY(sparse_dims(nrows, ncols, d, I, J, k, p, D, m, Jm));
  if (R > (1LL << 31) - 1) return TNR_ERANGE;
  D.R = R;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t K = D.K, olen = omega_len(Jm, K);
  Arena ar;
  ar.base = static_cast<char *>(ws);
  ar.size = ws_bytes;
  SBufs b;
  carve_sparse(ar, D, R, olen, b);
  int64_t *dims = ar.take<int64_t>(2 * TNR_MAX_SITES);
  if (!ar.ok || !dims) return TNR_ENOMEM;
  TNR_TRY(reset_status(s));
  // block rows / columns, then compact row and column lists of the nonzeros (built once per call)
  {
    std::vector<int64_t> h(2 * TNR_MAX_SITES, 1);
    for (int i = 0; i < d; ++i) {
      h[i] = I[i];
      h[TNR_MAX_SITES + i] = J[i];
    }
    TNR_CK(cudaMemcpyAsync(dims, h.data(), sizeof(int64_t) * 2 * TNR_MAX_SITES, cudaMemcpyHostToDevice, s));
    if (d > 1) {
      LaunchScope ls(K_MISC, s);
      k_block_pq<<<grid_n(R), 256, 0, s>>>(digits, R, d - 1, dims, dims + TNR_MAX_SITES, b.p, b.q, status_ptr());
    } else {  // one block row and one block column
      TNR_CK(cudaMemsetAsync(b.p, 0, sizeof(int) * R, s));
      TNR_CK(cudaMemsetAsync(b.q, 0, sizeof(int) * R, s));
    }
  }
  TNR_CK(cudaGetLastError());
  for (int by_col = 0; by_col < 2; ++by_col) {
    const int64_t n = by_col ? D.ncols : D.nrows;
    int *cnt = by_col ? b.ccnt : b.rcnt, *ptr = by_col ? b.cptr : b.rptr, *idx = by_col ? b.cidx : b.ridx;
    double *val = by_col ? b.cval : b.rval;
    TNR_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
    LaunchScope ls(K_MISC, s);
    k_nz_count<<<grid_n(R * D.I1 * D.J1), 256, 0, s>>>(X, b.p, b.q, R, D.I1, D.J1, by_col, cnt);
    const int64_t tiles = cdiv(n, kScanTile);
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(cnt, n, ptr, b.tiles);
    k_scan_small<<<1, 1024, 0, s>>>(b.tiles, tiles, ptr + n);
    k_scan_add<<<grid_n(n), 256, 0, s>>>(ptr, n, b.tiles);
    TNR_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
    k_nz_fill<<<grid_n(R * D.I1 * D.J1), 256, 0, s>>>(X, b.p, b.q, R, D.I1, D.J1, by_col, ptr, cnt, idx, val);
    k_sort_lists<<<grid_n(n), 256, 0, s>>>(ptr, n, idx, val);
  }
  TNR_CK(cudaGetLastError());
  // Omega (Lemma 5.1 over the merged column dims), dense
  TNR_TRY(omega_fill(s, seed, olen, b.draws));
  {
    std::vector<int64_t> h(Jm.begin(), Jm.end());
    h.resize(TNR_MAX_SITES, 1);
    TNR_CK(cudaMemcpyAsync(dims, h.data(), sizeof(int64_t) * TNR_MAX_SITES, cudaMemcpyHostToDevice, s));
    LaunchScope ls(K_OMEGA, s);
    k_omega_dense<<<grid_n(D.ncols * K), 256, 0, s>>>(b.draws, (int)Jm.size(), dims, K, D.ncols, b.O);
  }
  TNR_CK(cudaGetLastError());
  const int64_t nr = D.nrows, nc = D.ncols;
  // Y = A Omega; Q = qr(Y); q times { Q = qr(A^T Q); Q = qr(A Q) }  (row-major tall matrices)
  int nnz = 0;
  TNR_CK(cudaMemcpyAsync(&nnz, b.rptr + nr, sizeof(int), cudaMemcpyDeviceToHost, s));
  TNR_TRY(read_status(s));
  TNR_TRY(spmm(s, b.rptr, b.ridx, b.rval, nr, nc, K, b.O, b.Q, nnz));
  TNR_TRY(chol_qr(s, b.Q, nr, K, b, false));
  for (int it = 0; it < q; ++it) {
    TNR_TRY(spmm(s, b.cptr, b.cidx, b.cval, nc, nr, K, b.Q, b.Z, nnz));
    TNR_TRY(chol_qr(s, b.Z, nc, K, b, false));
    TNR_TRY(spmm(s, b.rptr, b.ridx, b.rval, nr, nc, K, b.Z, b.Q, nnz));
    TNR_TRY(chol_qr(s, b.Q, nr, K, b, false));
  }
  // B^T = Z = A^T Q; Z = Qz Rz; SVD of Rz^T = W S Zr^T; U = Q W, V = Qz Zr
  TNR_TRY(spmm(s, b.cptr, b.cidx, b.cval, nc, nr, K, b.Q, b.Z, nnz));
  TNR_TRY(chol_qr(s, b.Z, nc, K, b, true));
  TNR_TRY(copy_matrix_f64(s, b.Racc, K, b.G, K, K, K, true));  // G = Rz^T
  TNR_TRY(jacobi_svd_f64(s, b.G, K, K, b.Sv, b.Vk, K, b.jac));  // G <- W, Sv, Vk = Zr
  // row-major Q (nr x K) is the column-major K x nr matrix Q^T
  TNR_TRY(gemm_f64(s, true, false, nr, k, K, 1.0, b.Q, K, 0, b.G, K, 0, 0.0, U, nr, 0));
  TNR_TRY(gemm_f64(s, true, false, nc, k, K, 1.0, b.Z, K, 0, b.Vk, K, 0, 0.0, V, nc, 0));
  TNR_CK(cudaMemcpyAsync(S, b.Sv, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  return read_status(s);
}
