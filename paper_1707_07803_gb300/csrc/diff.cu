// Differentiable TNrSVD: a forward that records every step (a tape) and its hand-written
// adjoint, giving the gradient of a loss of the returned singular values with respect to the
// cores of A.
//
// The forward is Alg. 5.4 feeding Alg. 5.1 (leading-site merge, Omega of Lemma 5.1, the 2q+2
// products of Section 5.2, the MPO-QR of Alg. 5.2 with the rounding sweeps of Section 5.4, the
// MPO-SVD of Alg. 5.3) in FP64 with fixed ranks: tol = 0 (only exactly-zero singular values are
// dropped) and max_rank = K, so that the map cores -> S is smooth where singular values are
// simple. No compression or no-truncation shortcut is taken here: each step is the literal step,
// and the tape keeps what its adjoint needs (per-site checkpoints of both sweeps).
//
// Adjoints (vector-Jacobian products), derived for the real case:
//   product Y = op(A) (x) X (Section 5.2): transposed contractions of Ybar with X and with A;
//   thin QR A = Q R (m >= n): Abar = (Qbar + Q copyltu(M)) R^{-T}, M = R Rbar^T - Qbar^T Q,
//     copyltu(M) = tril(M) + tril(M, -1)^T; for m < n the trailing columns Y = Q R2 give
//     Ybar = Q R2bar and the square factor sees Qbar + Y R2bar^T;
//   thin SVD A = U S V^T (all k = min(m, n) values, the kept ones and the truncated ones, so the
//     gaps between kept and dropped values enter through F):
//     Abar = U [F o (U^T Ubar - Ubar^T U) S + S F o (V^T Vbar - Vbar^T V) + diag(Sbar)] V^T
//            + (I - U U^T) Ubar S^{-1} V^T + U S^{-1} Vbar^T (I - V V^T),  F_ij = 1/(s_j^2 - s_i^2);
//   absorbs C' = C (U S), C' = R C: plain GEMM adjoints; merge: transposed contractions.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tnr_internal.cuh"

namespace tnr {
namespace {

constexpr int kMaxO = 6, kMaxS = 4;

// ---- generic strided contraction: O[o] = sum_s X[x(o, s)] * Y[y(o, s)] (+ beta O[o]) --------------
struct GSpec {
  int no, ns;
  int64_t osz[kMaxO], ox[kMaxO], oy[kMaxO], oo[kMaxO];
  int64_t ssz[kMaxS], sx[kMaxS], sy[kMaxS];
  int64_t nout, nsum;
  double beta;
};

__global__ void k_gcontract(const double *__restrict__ X, const double *__restrict__ Y, double *O, GSpec g) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < g.nout; o += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = o, px = 0, py = 0, po = 0;
    for (int d = 0; d < g.no; ++d) {
      const int64_t v = rem % g.osz[d];
      rem /= g.osz[d];
      px += v * g.ox[d];
      py += v * g.oy[d];
      po += v * g.oo[d];
    }
    double acc = 0.0;
    int64_t idx[kMaxS] = {0, 0, 0, 0};
    for (int64_t s = 0; s < g.nsum; ++s) {
      acc = fma(X[px], Y ? Y[py] : 1.0, acc);
      for (int d = 0; d < g.ns; ++d) {
        px += g.sx[d];
        py += g.sy[d];
        if (++idx[d] < g.ssz[d]) break;
        px -= g.sx[d] * g.ssz[d];
        py -= g.sy[d] * g.ssz[d];
        idx[d] = 0;
      }
    }
    O[po] = g.beta == 0.0 ? acc : fma(g.beta, O[po], acc);
  }
}

struct Dim {
  int64_t size, sx, sy, so;
};

int gcontract(cudaStream_t s, const double *X, const double *Y, double *O, std::initializer_list<Dim> out,
              std::initializer_list<Dim> sum, double beta) {
  GSpec g;
  memset(&g, 0, sizeof(g));
  g.no = 0;
  g.nout = 1;
  for (const Dim &d : out) {
    if (d.size <= 0) return TNR_OK;
    g.osz[g.no] = d.size;
    g.ox[g.no] = d.sx;
    g.oy[g.no] = d.sy;
    g.oo[g.no] = d.so;
    g.nout *= d.size;
    ++g.no;
  }
  g.ns = 0;
  g.nsum = 1;
  for (const Dim &d : sum) {
    if (d.size <= 0) return TNR_OK;
    g.ssz[g.ns] = d.size;
    g.sx[g.ns] = d.sx;
    g.sy[g.ns] = d.sy;
    g.nsum *= d.size;
    ++g.ns;
  }
  g.beta = beta;
  const int64_t blocks = std::min<int64_t>(cdiv(g.nout, 256), 65536);
  LaunchScope ls(K_DIFF, s);
  k_gcontract<<<(unsigned)blocks, 256, 0, s>>>(X, Y, O, g);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// ---- small element-wise kernels ----------------------------------------------------------------
// B (m x n, ld m) = A (ld lda), optionally transposed (B = A^T, A is n x m)
__global__ void k_copy_t(const double *A, int64_t lda, double *B, int64_t m, int64_t n, int trans) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = t / m;
    B[t] = trans ? A[j + lda * i] : A[i + lda * j];
  }
}

// M (n x n) <- copyltu(M) = tril(M) + tril(M, -1)^T
__global__ void k_copyltu(double *M, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    if (i < j) M[t] = M[j + n * i];
  }
}

// X (m x n) <- B R^{-T} for R upper triangular (n x n, ld ldr): row by row, x R^T = b is solved by
// back substitution from the last column (x_j = (b_j - sum_{l>j} R_jl x_l) / R_jj).
__global__ void k_trsm_rt(double *B, int64_t m, int64_t n, const double *R, int64_t ldr, int *status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t j = n - 1; j >= 0; --j) {
      double acc = B[i + m * j];
      for (int64_t l = j + 1; l < n; ++l) acc = fma(-R[j + ldr * l], B[i + m * l], acc);
      const double dj = R[j + ldr * j];
      if (dj == 0.0) {
        set_status(status, TNR_ENONFINITE);
        acc = 0.0;
      } else {
        acc /= dj;
      }
      B[i + m * j] = acc;
    }
  }
}

// J (k x k) from A = U^T Ubar, B = V^T Vbar, singular values s and Sbar (see the file comment)
__global__ void k_svd_middle(const double *A, const double *B, const double *s, const double *gs, double *J, int64_t k) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % k, j = t / k;
    if (i == j) {
      J[t] = gs[i];
    } else {
      const double den = s[j] * s[j] - s[i] * s[i];
      const double f = den != 0.0 ? 1.0 / den : 0.0;  // equal values: no defined rotation (zero term)
      J[t] = f * (A[i + k * j] - A[j + k * i]) * s[j] + s[i] * f * (B[i + k * j] - B[j + k * i]);
    }
  }
}

// C (m x n) = A (m x n, ld lda) diag(d^p), p = +1 or -1 (columns scaled)
__global__ void k_scale_by(const double *A, int64_t lda, double *C, int64_t m, int64_t n, const double *d, int inv) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = t / m;
    C[t] = inv ? (d[j] != 0.0 ? A[i + lda * j] / d[j] : 0.0) : A[i + lda * j] * d[j];
  }
}

// g[j] = sum_i U[i, j] * G[i, j] for j < r, 0 for r <= j < n
__global__ void k_coldots(const double *U, int64_t ldu, const double *G, int64_t ldg, int64_t m, int64_t r, int64_t n,
                          double *g) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (j < r)
      for (int64_t i = 0; i < m; ++i) acc = fma(U[i + ldu * j], G[i + ldg * j], acc);
    g[j] = acc;
  }
}

__global__ void k_axpy(const double *x, double *y, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) y[t] += x[t];
}

int grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 65536)); }

// ---- device memory owned by a tape or by one call ---------------------------------------------
struct Pool {
  cudaStream_t s = nullptr;
  std::vector<void *> ptrs;
  bool ok = true;
  double *take(int64_t n) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, sizeof(double) * (size_t)std::max<int64_t>(n, 1), s) != cudaSuccess) {
      ok = false;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<double *>(p);
  }
  void release() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
    ptrs.clear();
  }
};

#define DTAKE(var, pool, n)                 \
  double *var = (pool).take(n);             \
  if (!var) return TNR_ENOMEM;

int copy_mat(cudaStream_t s, const double *A, int64_t lda, double *B, int64_t m, int64_t n, bool trans) {
  if (m <= 0 || n <= 0) return TNR_OK;
  LaunchScope ls(K_DIFF, s);
  k_copy_t<<<grid(m * n), 256, 0, s>>>(A, lda, B, m, n, trans ? 1 : 0);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

int zero(cudaStream_t s, double *x, int64_t n) {
  if (n <= 0) return TNR_OK;
  TNR_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  return TNR_OK;
}

// C (m x n) = op(A) op(B) (+ beta C), column-major, packed leading dimensions unless given
int mm(cudaStream_t s, bool ta, bool tb, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
       const double *B, int64_t ldb, double beta, double *C, int64_t ldc) {
  if (m <= 0 || n <= 0) return TNR_OK;
  if (k <= 0) return beta == 0.0 ? zero(s, C, m * n) : TNR_OK;
  return gemm_f64(s, ta, tb, m, n, k, 1.0, A, lda, 0, B, ldb, 0, beta, C, ldc, 0);
}

// explicit thin QR: A (m x n) <- Q (m x q), R (q x n), q = min(m, n)
int thin_qr(cudaStream_t s, double *A, int64_t m, int64_t n, double *R, Pool &tmp) {
  const int64_t q = std::min(m, n);
  if (qr_small_fits(m, n))
    return qr_small_f64(s, A, m, m, n, false, false, 0.0, A, m, false, R, q, false, nullptr);
  DTAKE(scr, tmp, (int64_t)(qr_f64_scratch(m, n) / sizeof(double)) + 1);
  return qr_f64(s, A, m, n, m, R, q, scr);
}

// full thin SVD of M (t x w): U (t x n), S (n), V (w x n), n = min(t, w), S descending
int full_svd(cudaStream_t s, const double *M, int64_t t, int64_t w, double *U, double *S, double *V, Pool &tmp) {
  const int64_t n = std::min(t, w);
  const size_t js = jacobi_scratch(n);
  double *jscr = js ? tmp.take((int64_t)(js / sizeof(double)) + 1) : nullptr;
  if (js && !jscr) return TNR_ENOMEM;
  DTAKE(Rm, tmp, n * n);
  DTAKE(G, tmp, n * n);
  DTAKE(Vr, tmp, n * n);
  if (t >= w) {
    DTAKE(Qm, tmp, t * w);
    TNR_TRY(copy_mat(s, M, t, Qm, t, w, false));
    TNR_TRY(thin_qr(s, Qm, t, w, Rm, tmp));  // M = Qm Rm
    TNR_TRY(copy_mat(s, Rm, n, G, n, n, false));
    TNR_TRY(jacobi_svd_f64(s, G, n, n, S, Vr, n, jscr));  // Rm = G S Vr^T
    TNR_TRY(mm(s, false, false, t, n, n, Qm, t, G, n, 0.0, U, t));
    TNR_TRY(copy_mat(s, Vr, n, V, w, n, false));
  } else {
    DTAKE(Qm, tmp, w * t);
    TNR_TRY(copy_mat(s, M, t, Qm, w, t, true));  // M^T (w x t)
    TNR_TRY(thin_qr(s, Qm, w, t, Rm, tmp));      // M^T = Qm Rm, M = Rm^T Qm^T
    TNR_TRY(copy_mat(s, Rm, n, G, n, n, true));  // G = Rm^T
    TNR_TRY(jacobi_svd_f64(s, G, n, n, S, Vr, n, jscr));  // Rm^T = G S Vr^T
    TNR_TRY(copy_mat(s, G, n, U, t, n, false));
    TNR_TRY(mm(s, false, false, w, n, n, Qm, w, Vr, n, 0.0, V, w));  // V = Qm Vr
  }
  return TNR_OK;
}

// Abar (m x n) of the thin QR A = Q R (Q m x q, R q x n, q = min(m, n)); gQ, gR may be null (zero)
int qr_vjp(cudaStream_t s, const double *Q, const double *R, const double *gQ, const double *gR, int64_t m,
           int64_t n, double *gA, Pool &tmp) {
  const int64_t q = std::min(m, n);
  DTAKE(gQe, tmp, m * q);  // effective Qbar of the square-or-tall factor
  if (gQ)
    TNR_TRY(copy_mat(s, gQ, m, gQe, m, q, false));
  else
    TNR_TRY(zero(s, gQe, m * q));
  DTAKE(gR1, tmp, q * q);
  if (gR)
    TNR_TRY(copy_mat(s, gR, q, gR1, q, q, false));
  else
    TNR_TRY(zero(s, gR1, q * q));
  if (n > q) {  // wide: A = [X Y], Y = Q R2
    const int64_t n2 = n - q;
    const double *R2 = R + q * q;
    // Ybar = Q R2bar  (into gA's trailing columns)
    if (gR)
      TNR_TRY(mm(s, false, false, m, n2, q, Q, m, gR + q * q, q, 0.0, gA + m * q, m));
    else
      TNR_TRY(zero(s, gA + m * q, m * n2));
    if (gR) {  // Qbar += Y R2bar^T with Y = Q R2
      DTAKE(Y, tmp, m * n2);
      TNR_TRY(mm(s, false, false, m, n2, q, Q, m, R2, q, 0.0, Y, m));
      TNR_TRY(mm(s, false, true, m, q, n2, Y, m, gR + q * q, q, 1.0, gQe, m));
    }
  }
  // square/tall part on the leading q columns: M = R1 R1bar^T - Qbar^T Q
  DTAKE(M, tmp, q * q);
  TNR_TRY(mm(s, false, true, q, q, q, R, q, gR1, q, 0.0, M, q));
  TNR_TRY(gemm_f64(s, true, false, q, q, m, -1.0, gQe, m, 0, Q, m, 0, 1.0, M, q, 0));  // M -= Qbar^T Q
  {
    LaunchScope ls(K_DIFF, s);
    k_copyltu<<<grid(q * q), 256, 0, s>>>(M, q);
  }
  TNR_CK(cudaGetLastError());
  // B = Qbar + Q copyltu(M)   (m x q), then B R1^{-T}
  DTAKE(B, tmp, m * q);
  TNR_TRY(copy_mat(s, gQe, m, B, m, q, false));
  TNR_TRY(mm(s, false, false, m, q, q, Q, m, M, q, 1.0, B, m));
  {
    LaunchScope ls(K_DIFF, s);
    k_trsm_rt<<<grid(m), 256, 0, s>>>(B, m, q, R, q, status_ptr());
  }
  TNR_CK(cudaGetLastError());
  return copy_mat(s, B, m, gA, m, q, false);
}

// Abar (m x n) of the thin SVD A = U S V^T (U m x k, V n x k, k = min(m, n)); gU (m x k), gS (k),
// gV (n x k) full-width (zero where not used)
int svd_vjp(cudaStream_t s, const double *U, const double *S, const double *V, const double *gU, const double *gS,
            const double *gV, int64_t m, int64_t n, double *gA, Pool &tmp) {
  const int64_t k = std::min(m, n);
  DTAKE(Au, tmp, k * k);
  DTAKE(Bv, tmp, k * k);
  DTAKE(J, tmp, k * k);
  TNR_TRY(mm(s, true, false, k, k, m, U, m, gU, m, 0.0, Au, k));
  TNR_TRY(mm(s, true, false, k, k, n, V, n, gV, n, 0.0, Bv, k));
  {
    LaunchScope ls(K_DIFF, s);
    k_svd_middle<<<grid(k * k), 256, 0, s>>>(Au, Bv, S, gS, J, k);
  }
  TNR_CK(cudaGetLastError());
  // G1 = U J + (I - U U^T) gU S^{-1}
  DTAKE(T1, tmp, m * k);
  {
    LaunchScope ls(K_DIFF, s);
    k_scale_by<<<grid(m * k), 256, 0, s>>>(gU, m, T1, m, k, S, 1);
  }
  TNR_CK(cudaGetLastError());
  DTAKE(P, tmp, k * k);
  TNR_TRY(mm(s, true, false, k, k, m, U, m, T1, m, 0.0, P, k));
  TNR_TRY(gemm_f64(s, false, false, m, k, k, -1.0, U, m, 0, P, k, 0, 1.0, T1, m, 0));
  TNR_TRY(mm(s, false, false, m, k, k, U, m, J, k, 1.0, T1, m));
  TNR_TRY(mm(s, false, true, m, n, k, T1, m, V, n, 0.0, gA, m));  // gA = G1 V^T
  // + U [(I - V V^T) gV S^{-1}]^T
  DTAKE(T2, tmp, n * k);
  {
    LaunchScope ls(K_DIFF, s);
    k_scale_by<<<grid(n * k), 256, 0, s>>>(gV, n, T2, n, k, S, 1);
  }
  TNR_CK(cudaGetLastError());
  TNR_TRY(mm(s, true, false, k, k, n, V, n, T2, n, 0.0, P, k));
  TNR_TRY(gemm_f64(s, false, false, n, k, k, -1.0, V, n, 0, P, k, 0, 1.0, T2, n, 0));
  return mm(s, false, true, m, n, k, U, m, T2, n, 1.0, gA, m);
}

// ---- products (Section 5.2) and their adjoints ---------------------------------------------
// core dims (r, x, c, r2) of a site; X-operand rows are y (= J of A without trans, I with trans)
struct Site {
  int64_t R, I, J, R2;
};

// Y((a, s), x, c, (a2, s2)) = sum_y A(a, ., ., a2) X(s, y, c, s2); x = i, y = j (no trans) or
// x = j, y = i (trans). A: (R, I, J, R2); X: (S, Ny, Kx, S2); Y: (R S, Nx, Kx, R2 S2).
int prod_fwd(cudaStream_t s, const double *A, Site a, int trans, const double *X, int64_t S, int64_t Kx, int64_t S2,
             double *Y) {
  const int64_t Nx = trans ? a.J : a.I, Ny = trans ? a.I : a.J;
  const int64_t ax = trans ? a.R * a.I : a.R, ay = trans ? a.R : a.R * a.I;  // A strides of x and y
  const int64_t RS = a.R * S;
  return gcontract(s, A, X, Y,
                   {{a.R, 1, 0, 1},
                    {S, 0, 1, a.R},
                    {Nx, ax, 0, RS},
                    {Kx, 0, S * Ny, RS * Nx},
                    {a.R2, a.R * a.I * a.J, 0, RS * Nx * Kx},
                    {S2, 0, S * Ny * Kx, RS * Nx * Kx * a.R2}},
                   {{Ny, ay, S, 0}}, 0.0);
}

// gA += contraction of gY with X;  gX += contraction of gY with A (gX may be null)
int prod_bwd(cudaStream_t s, const double *A, Site a, int trans, const double *X, int64_t S, int64_t Kx, int64_t S2,
             const double *gY, double *gA, double *gX) {
  const int64_t Nx = trans ? a.J : a.I, Ny = trans ? a.I : a.J;
  const int64_t RS = a.R * S;
  // gA(a, i, j, a2): i and j are x / y in the order given by trans
  const int64_t gy_i = trans ? 0 : RS, gy_j = trans ? RS : 0;  // gY strides of i and j (x only)
  const int64_t x_i = trans ? S : 0, x_j = trans ? 0 : S;      // X strides of i and j (y only)
  TNR_TRY(gcontract(s, gY, X, gA,
                    {{a.R, 1, 0, 1}, {a.I, gy_i, x_i, a.R}, {a.J, gy_j, x_j, a.R * a.I},
                     {a.R2, RS * Nx * Kx, 0, a.R * a.I * a.J}},
                    {{S, a.R, 1, 0}, {Kx, RS * Nx, S * Ny, 0}, {S2, RS * Nx * Kx * a.R2, S * Ny * Kx, 0}}, 1.0));
  if (!gX) return TNR_OK;
  const int64_t ax = trans ? a.R * a.I : a.R, ay = trans ? a.R : a.R * a.I;
  return gcontract(s, gY, A, gX,
                   {{S, a.R, 0, 1}, {Ny, 0, ay, S}, {Kx, RS * Nx, 0, S * Ny}, {S2, RS * Nx * Kx * a.R2, 0, S * Ny * Kx}},
                   {{a.R, 1, 1, 0}, {Nx, RS, ax, 0}, {a.R2, RS * Nx * Kx, a.R * a.I * a.J, 0}}, 1.0);
}

// merge of two leading cores: M (1, I0 I1, J0 J1, R2) = A0 (1, I0, J0, R1) . A1 (R1, I1, J1, R2)
int merge_fwd(cudaStream_t s, const double *A0, int64_t I0, int64_t J0, const double *A1, Site b, double *M) {
  const int64_t II = I0 * b.I, JJ = J0 * b.J;
  return gcontract(s, A0, A1, M,
                   {{I0, 1, 0, 1}, {b.I, 0, b.R, I0}, {J0, I0, 0, II}, {b.J, 0, b.R * b.I, II * J0},
                    {b.R2, 0, b.R * b.I * b.J, II * JJ}},
                   {{b.R, I0 * J0, 1, 0}}, 0.0);
}

int merge_bwd(cudaStream_t s, const double *A0, int64_t I0, int64_t J0, const double *A1, Site b, const double *gM,
              double *gA0, double *gA1) {
  const int64_t II = I0 * b.I, JJ = J0 * b.J;
  TNR_TRY(gcontract(s, gM, A1, gA0, {{I0, 1, 0, 1}, {J0, II, 0, I0}, {b.R, 0, 1, I0 * J0}},
                    {{b.I, I0, b.R, 0}, {b.J, II * J0, b.R * b.I, 0}, {b.R2, II * JJ, b.R * b.I * b.J, 0}}, 1.0));
  return gcontract(s, gM, A0, gA1,
                   {{b.R, 0, I0 * J0, 1}, {b.I, I0, 0, b.R}, {b.J, II * J0, 0, b.R * b.I},
                    {b.R2, II * JJ, 0, b.R * b.I * b.J}},
                   {{I0, 1, 1, 0}, {J0, II, I0, 0}}, 1.0);
}

// site-1 permutation: core (1, I1, K, t) <-> matrix A1^T ((I1 t) x K), (i + I1 r, c) <-> (i, c, r)
int site1_to_mat(cudaStream_t s, const double *core, int64_t I1, int64_t K, int64_t t, double *mat, double beta) {
  return gcontract(s, core, nullptr, mat, {{I1, 1, 0, 1}, {t, I1 * K, 0, I1}, {K, I1, 0, I1 * t}}, {}, beta);
}
int mat_to_site1(cudaStream_t s, const double *mat, int64_t I1, int64_t K, int64_t t, double *core, double beta) {
  return gcontract(s, mat, nullptr, core, {{I1, 1, 0, 1}, {K, I1 * t, 0, I1}, {t, I1, 0, I1 * K}}, {}, beta);
}

// ---- one MPO-QR (Alg. 5.2) or MPO-SVD (Alg. 5.3) with the rounding sweeps, on the tape ---------
struct OrthRec {
  bool svd = false;
  int d = 0;
  int64_t K = 0, I1 = 0;
  int64_t phys[TNR_MAX_SITES];  // row multiplicity of core k: I_k for k >= 1, I_1 K for k = 0
  int64_t Rin[TNR_MAX_SITES + 1], Rlr[TNR_MAX_SITES + 1], Rrl[TNR_MAX_SITES + 1];
  const double *Cin[TNR_MAX_SITES];
  double *Qlr[TNR_MAX_SITES], *Rf[TNR_MAX_SITES];
  double *M[TNR_MAX_SITES], *U[TNR_MAX_SITES], *S[TNR_MAX_SITES], *V[TNR_MAX_SITES];
  int64_t n[TNR_MAX_SITES];
  double *P0 = nullptr, *Qt = nullptr, *Rt = nullptr, *W = nullptr, *Sf = nullptr, *Zr = nullptr;
  double *out[TNR_MAX_SITES];
};

// Y: cores Cin (ranks Rin), site dims I (rows) with K columns on site 1. Fills rec and rec.out.
int orth_fwd(cudaStream_t s, OrthRec &rec, Pool &tape, Pool &tmp) {
  const int d = rec.d;
  const int64_t K = rec.K;
  rec.Rlr[0] = 1;
  rec.Rrl[0] = 1;
  rec.Rrl[d] = 1;
  rec.Rlr[d] = 1;
  // left-to-right QR sweep
  const double *cur = rec.Cin[0];
  int64_t curR = 1;  // left rank of the current core
  for (int k = 0; k + 1 < d; ++k) {
    const int64_t rows = curR * rec.phys[k], cols = rec.Rin[k + 1], q = std::min(rows, cols);
    const int64_t w1 = rec.phys[k + 1] * rec.Rin[k + 2];
    double *Qk = tape.take(rows * std::max(cols, q));
    double *Rk = tape.take(q * cols);
    double *next = tape.take(q * w1);
    if (!Qk || !Rk || !next) return TNR_ENOMEM;
    TNR_TRY(copy_mat(s, cur, rows, Qk, rows, cols, false));
    TNR_TRY(thin_qr(s, Qk, rows, cols, Rk, tmp));
    TNR_TRY(mm(s, false, false, q, w1, cols, Rk, q, rec.Cin[k + 1], cols, 0.0, next, q));
    rec.Qlr[k] = Qk;
    rec.Rf[k] = Rk;
    rec.Rlr[k + 1] = q;
    cur = next;
    curR = q;
  }
  rec.Qlr[d - 1] = const_cast<double *>(cur);
  rec.Rf[d - 1] = nullptr;
  // right-to-left truncating SVD sweep (tol = 0, ranks <= K)
  const double *Mk = rec.Qlr[d - 1];
  for (int k = d - 1; k >= 1; --k) {
    const int64_t t = rec.Rlr[k], w = rec.phys[k] * rec.Rrl[k + 1], n = std::min(t, w);
    double *U = tape.take(t * n), *S = tape.take(n), *V = tape.take(w * n);
    if (!U || !S || !V) return TNR_ENOMEM;
    TNR_TRY(full_svd(s, Mk, t, w, U, S, V, tmp));
    std::vector<double> hs(n);
    TNR_CK(cudaMemcpyAsync(hs.data(), S, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    TNR_TRY(read_status(s));
    int64_t r = 0;
    while (r < n && hs[r] > 0.0) ++r;  // tol = 0: only exact zeros are dropped
    r = std::max<int64_t>(1, std::min(r, K));
    rec.M[k] = const_cast<double *>(Mk);
    rec.U[k] = U;
    rec.S[k] = S;
    rec.V[k] = V;
    rec.n[k] = n;
    rec.Rrl[k] = r;
    double *ok = tape.take(r * w);
    if (!ok) return TNR_ENOMEM;
    TNR_TRY(copy_mat(s, V, w, ok, r, w, true));  // V[:, :r]^T
    rec.out[k] = ok;
    // core k-1 <- Qlr[k-1] (U S)
    DTAKE(US, tmp, t * r);
    {
      LaunchScope ls(K_DIFF, s);
      k_scale_by<<<grid(t * r), 256, 0, s>>>(U, t, US, t, r, S, 0);
    }
    TNR_CK(cudaGetLastError());
    const int64_t rows = rec.Rlr[k - 1] * rec.phys[k - 1];
    double *nm = tape.take(rows * r);
    if (!nm) return TNR_ENOMEM;
    TNR_TRY(mm(s, false, false, rows, r, t, rec.Qlr[k - 1], rows, US, t, 0.0, nm, rows));
    Mk = nm;
  }
  rec.P0 = const_cast<double *>(Mk);  // core 0: (1, I1, K, r1)
  const int64_t r1 = d > 1 ? rec.Rrl[1] : rec.Rin[1];
  const int64_t m = rec.I1 * r1;
  if (m < K) return TNR_EINVAL;
  rec.Qt = tape.take(m * K);
  rec.Rt = tape.take(K * K);
  if (!rec.Qt || !rec.Rt) return TNR_ENOMEM;
  TNR_TRY(site1_to_mat(s, rec.P0, rec.I1, K, r1, rec.Qt, 0.0));
  TNR_TRY(thin_qr(s, rec.Qt, m, K, rec.Rt, tmp));  // A1^T = Qt Rt
  double *o0 = tape.take(m * K);
  if (!o0) return TNR_ENOMEM;
  if (!rec.svd) {
    TNR_TRY(mat_to_site1(s, rec.Qt, rec.I1, K, r1, o0, 0.0));
  } else {  // R^T = W S Zr^T: W, S (descending), V^(1) = Qt Zr
    rec.W = tape.take(K * K);
    rec.Sf = tape.take(K);
    rec.Zr = tape.take(K * K);
    if (!rec.W || !rec.Sf || !rec.Zr) return TNR_ENOMEM;
    TNR_TRY(copy_mat(s, rec.Rt, K, rec.W, K, K, true));
    const size_t js = jacobi_scratch(K);
    double *jscr = js ? tmp.take((int64_t)(js / sizeof(double)) + 1) : nullptr;
    if (js && !jscr) return TNR_ENOMEM;
    TNR_TRY(jacobi_svd_f64(s, rec.W, K, K, rec.Sf, rec.Zr, K, jscr));
    DTAKE(QZ, tmp, m * K);
    TNR_TRY(mm(s, false, false, m, K, K, rec.Qt, m, rec.Zr, K, 0.0, QZ, m));
    TNR_TRY(mat_to_site1(s, QZ, rec.I1, K, r1, o0, 0.0));
  }
  rec.out[0] = o0;
  return TNR_OK;
}

// adjoint of orth_fwd: gOut[k] (grads of rec.out[k], null = zero; MPO-SVD: ignored), gSf (MPO-SVD
// only: K values, grads of Sf). Writes gCin[k] (grads of the input cores, caller-zeroed buffers).
int orth_bwd(cudaStream_t s, const OrthRec &rec, double *const *gOut, const double *gSf, double *const *gCin,
             Pool &tmp) {
  const int d = rec.d;
  const int64_t K = rec.K;
  const int64_t r1 = d > 1 ? rec.Rrl[1] : rec.Rin[1];
  const int64_t m = rec.I1 * r1;
  // site 1
  DTAKE(gQt, tmp, m * K);
  DTAKE(gRt, tmp, K * K);
  if (!rec.svd) {
    if (gOut && gOut[0])
      TNR_TRY(site1_to_mat(s, gOut[0], rec.I1, K, r1, gQt, 0.0));
    else
      TNR_TRY(zero(s, gQt, m * K));
    TNR_TRY(zero(s, gRt, K * K));
  } else {
    TNR_TRY(zero(s, gQt, m * K));
    // d(R^T) = W diag(gS) Zr^T  ->  gRt = Zr diag(gS) W^T
    DTAKE(ZS, tmp, K * K);
    {
      LaunchScope ls(K_DIFF, s);
      k_scale_by<<<grid(K * K), 256, 0, s>>>(rec.Zr, K, ZS, K, K, gSf, 0);
    }
    TNR_CK(cudaGetLastError());
    TNR_TRY(mm(s, false, true, K, K, K, ZS, K, rec.W, K, 0.0, gRt, K));
  }
  DTAKE(gA1t, tmp, m * K);
  TNR_TRY(qr_vjp(s, rec.Qt, rec.Rt, gQt, gRt, m, K, gA1t, tmp));
  const int64_t rows0 = rec.phys[0];
  DTAKE(gX, tmp, rows0 * r1);
  TNR_TRY(mat_to_site1(s, gA1t, rec.I1, K, r1, gX, 0.0));
  // right-to-left sweep, in reverse (k = 1 .. d-1)
  std::vector<double *> gQlr(d, nullptr);
  double *gM = gX;  // grad of core k-1 after step k
  for (int k = 1; k < d; ++k) {
    const int64_t t = rec.Rlr[k], r = rec.Rrl[k], w = rec.phys[k] * rec.Rrl[k + 1], n = rec.n[k];
    const int64_t rows = rec.Rlr[k - 1] * rec.phys[k - 1];
    DTAKE(US, tmp, t * r);
    {
      LaunchScope ls(K_DIFF, s);
      k_scale_by<<<grid(t * r), 256, 0, s>>>(rec.U[k], t, US, t, r, rec.S[k], 0);
    }
    TNR_CK(cudaGetLastError());
    // core_{k-1}' = Qlr[k-1] US
    gQlr[k - 1] = tmp.take(rows * t);
    if (!gQlr[k - 1]) return TNR_ENOMEM;
    TNR_TRY(mm(s, false, true, rows, t, r, gM, rows, US, t, 0.0, gQlr[k - 1], rows));
    DTAKE(gUS, tmp, t * r);
    TNR_TRY(mm(s, true, false, t, r, rows, rec.Qlr[k - 1], rows, gM, rows, 0.0, gUS, t));
    // SVD adjoint inputs, full width n (zero beyond r)
    DTAKE(gU, tmp, t * n);
    DTAKE(gS, tmp, n);
    DTAKE(gV, tmp, w * n);
    TNR_TRY(zero(s, gU, t * n));
    TNR_TRY(zero(s, gV, w * n));
    {
      LaunchScope ls(K_DIFF, s);
      k_scale_by<<<grid(t * r), 256, 0, s>>>(gUS, t, gU, t, r, rec.S[k], 0);  // Ubar = (US)bar S
      k_coldots<<<grid(n), 256, 0, s>>>(rec.U[k], t, gUS, t, t, r, n, gS);   // Sbar_j = u_j . (US)bar_j
    }
    TNR_CK(cudaGetLastError());
    if (gOut && gOut[k] && !rec.svd) TNR_TRY(copy_mat(s, gOut[k], r, gV, w, r, true));  // Vbar = (V^T)bar^T
    double *gMk = tmp.take(t * w);
    if (!gMk) return TNR_ENOMEM;
    TNR_TRY(svd_vjp(s, rec.U[k], rec.S[k], rec.V[k], gU, gS, gV, t, w, gMk, tmp));
    gM = gMk;
  }
  // left-to-right sweep, in reverse: gM is the grad of the last core after the LR sweep
  double *gNext = gM;
  for (int k = d - 2; k >= 0; --k) {
    const int64_t rows = rec.Rlr[k] * rec.phys[k], cols = rec.Rin[k + 1], q = rec.Rlr[k + 1];
    const int64_t w1 = rec.phys[k + 1] * rec.Rin[k + 2];
    // C^pre_{k+1} = Rf[k] Cin[k+1]
    DTAKE(gR, tmp, q * cols);
    TNR_TRY(mm(s, false, true, q, cols, w1, gNext, q, rec.Cin[k + 1], cols, 0.0, gR, q));
    TNR_TRY(mm(s, true, false, cols, w1, q, rec.Rf[k], q, gNext, q, 1.0, gCin[k + 1], cols));
    double *gC = tmp.take(rows * cols);
    if (!gC) return TNR_ENOMEM;
    TNR_TRY(qr_vjp(s, rec.Qlr[k], rec.Rf[k], gQlr[k], gR, rows, cols, gC, tmp));
    gNext = gC;
  }
  // gNext: grad of C^pre_0 = Cin[0]
  const int64_t n0 = rec.phys[0] * rec.Rin[1];
  LaunchScope ls(K_DIFF, s);
  k_axpy<<<grid(n0), 256, 0, s>>>(gNext, gCin[0], n0);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

}  // namespace

// ---- the tape of one differentiable solve --------------------------------------------------
struct DiffTape {
  Pool mem;
  int d = 0, m = 0;  // merged sites, merge count
  int64_t K = 0, k = 0, p = 0, q = 0;
  tnr_mpo A;  // caller's operator (pointers only)
  int64_t Im[TNR_MAX_SITES], Jm[TNR_MAX_SITES], RA[TNR_MAX_SITES + 1];
  double *merged[TNR_MAX_SITES];  // merged[j] = cores 0..j merged (j = 1 .. m-1); merged[m-1] = site 1 of A'
  double *omega = nullptr;
  std::vector<OrthRec> recs;  // 2q + 2 records: Y, then (Z, Y) q times, then the MPO-SVD
  std::vector<std::vector<double *>> prods;  // the product cores fed to each record
};

}  // namespace tnr

using tnr::DiffTape;

namespace {

const double *site_core(const DiffTape &T, int k) { return k == 0 ? T.merged[T.m - 1] : T.A.core[T.m - 1 + k]; }
tnr::Site site_dims(const DiffTape &T, int k) { return {T.RA[k], T.Im[k], T.Jm[k], T.RA[k + 1]}; }

// product op(A') (x) X where X has ranks XR, K columns on site 1; output into a new record's inputs
int run_product(cudaStream_t s, DiffTape &T, int trans, const double *const *X, const int64_t *XR,
                tnr::OrthRec &rec) {
  const int d = T.d;
  rec.d = d;
  rec.K = T.K;
  rec.I1 = trans ? T.Jm[0] : T.Im[0];
  std::vector<double *> cores(d, nullptr);
  for (int k = 0; k < d; ++k) {
    const tnr::Site a = site_dims(T, k);
    const int64_t S = XR[k], S2 = XR[k + 1], Kx = k == 0 ? T.K : 1;
    const int64_t Nx = trans ? a.J : a.I;
    double *Y = T.mem.take(a.R * S * Nx * Kx * a.R2 * S2);
    if (!Y) return TNR_ENOMEM;
    TNR_TRY(tnr::prod_fwd(s, site_core(T, k), a, trans, X[k], S, Kx, S2, Y));
    cores[k] = Y;
    rec.Cin[k] = Y;
    rec.Rin[k] = a.R * S;
    rec.phys[k] = Nx * Kx;
  }
  rec.Rin[d] = 1;
  T.prods.push_back(cores);
  return TNR_OK;
}

int diff_forward(cudaStream_t s, DiffTape &T, uint64_t seed, double *S_out) {
  using namespace tnr;
  Pool tmp;
  tmp.s = s;
  const int d = T.d;
  // merged site 1 (Section 6.3), with every partial merge kept for the adjoint
  T.merged[0] = const_cast<double *>(T.A.core[0]);
  {
    int64_t I0 = T.A.I[0], J0 = T.A.J[0];
    for (int j = 1; j < T.m; ++j) {
      const Site b{T.A.R[j], T.A.I[j], T.A.J[j], T.A.R[j + 1]};
      double *M = T.mem.take(I0 * b.I * J0 * b.J * b.R2);
      if (!M) return TNR_ENOMEM;
      TNR_TRY(merge_fwd(s, T.merged[j - 1], I0, J0, T.A.core[j], b, M));
      T.merged[j] = M;
      I0 *= b.I;
      J0 *= b.J;
    }
  }
  // Omega (Lemma 5.1): site 1 (J1 x K, column-major), then one vector per site
  int64_t olen = T.Jm[0] * T.K;
  for (int k = 1; k < d; ++k) olen += T.Jm[k];
  T.omega = T.mem.take(olen);
  if (!T.omega) return TNR_ENOMEM;
  TNR_TRY(omega_fill(s, seed, olen, T.omega));
  std::vector<const double *> Om(d);
  std::vector<int64_t> OR(d + 1, 1);
  {
    int64_t pos = 0;
    for (int k = 0; k < d; ++k) {
      Om[k] = T.omega + pos;
      pos += k == 0 ? T.Jm[0] * T.K : T.Jm[k];
    }
  }
  const int nrec = 2 * (int)T.q + 2;
  T.recs.assign(nrec, OrthRec());
  auto fwd = [&](int i, int trans, const double *const *X, const int64_t *XR, bool svd) -> int {
    OrthRec &rec = T.recs[i];
    TNR_TRY(run_product(s, T, trans, X, XR, rec));
    rec.svd = svd;
    int rc = orth_fwd(s, rec, T.mem, tmp);
    tmp.release();
    return rc;
  };
  TNR_TRY(fwd(0, 0, Om.data(), OR.data(), false));
  for (int it = 0; it < (int)T.q; ++it) {
    const OrthRec &prev = T.recs[2 * it];
    TNR_TRY(fwd(2 * it + 1, 1, prev.out, prev.Rrl, false));
    const OrthRec &z = T.recs[2 * it + 1];
    TNR_TRY(fwd(2 * it + 2, 0, z.out, z.Rrl, false));
  }
  const OrthRec &last = T.recs[2 * T.q];
  TNR_TRY(fwd(nrec - 1, 1, last.out, last.Rrl, true));
  TNR_CK(cudaMemcpyAsync(S_out, T.recs[nrec - 1].Sf, sizeof(double) * T.k, cudaMemcpyDeviceToDevice, s));
  TNR_TRY(read_status(s));
  return tmp.ok ? TNR_OK : TNR_ENOMEM;
}

int diff_backward(cudaStream_t s, DiffTape &T, const double *dS, tnr_mpo *dA) {
  using namespace tnr;
  Pool tmp;
  tmp.s = s;
  const int d = T.d;
  const int nrec = (int)T.recs.size();
  // gradient of the merged operator's cores (site 1 of A' separately)
  std::vector<double *> gAm(d, nullptr);
  for (int k = 0; k < d; ++k) {
    const Site a = site_dims(T, k);
    gAm[k] = k == 0 ? tmp.take(a.R * a.I * a.J * a.R2) : dA->core[T.m - 1 + k];
    if (!gAm[k]) return TNR_ENOMEM;
    TNR_TRY(zero(s, gAm[k], a.R * a.I * a.J * a.R2));
  }
  DTAKE(gSf, tmp, T.K);
  TNR_TRY(zero(s, gSf, T.K));
  TNR_CK(cudaMemcpyAsync(gSf, dS, sizeof(double) * T.k, cudaMemcpyDeviceToDevice, s));
  std::vector<double *> gOut;  // grads of the cores the current record produced (null: none)
  for (int i = nrec - 1; i >= 0; --i) {
    const OrthRec &rec = T.recs[i];
    std::vector<double *> gIn(d, nullptr);
    for (int k = 0; k < d; ++k) {
      const int64_t n = rec.Rin[k] * rec.phys[k] * rec.Rin[k + 1];
      gIn[k] = tmp.take(n);
      if (!gIn[k]) return TNR_ENOMEM;
      TNR_TRY(zero(s, gIn[k], n));
    }
    TNR_TRY(orth_bwd(s, rec, gOut.empty() ? nullptr : gOut.data(), rec.svd ? gSf : nullptr, gIn.data(), tmp));
    // the product that fed this record: op(A') (x) X, X = previous record's output (or Omega)
    const int trans = (i == 0) ? 0 : ((i % 2 == 1 || i == nrec - 1) ? 1 : 0);
    const OrthRec *prev = i > 0 ? &T.recs[i - 1] : nullptr;
    std::vector<double *> gX(d, nullptr);
    for (int k = 0; k < d; ++k) {
      const Site a = site_dims(T, k);
      const int64_t S = prev ? prev->Rrl[k] : 1, S2 = prev ? prev->Rrl[k + 1] : 1, Kx = k == 0 ? T.K : 1;
      const int64_t Ny = trans ? a.I : a.J;
      const double *X;
      if (prev) {
        X = prev->out[k];
        gX[k] = tmp.take(S * Ny * Kx * S2);
        if (!gX[k]) return TNR_ENOMEM;
        TNR_TRY(zero(s, gX[k], S * Ny * Kx * S2));
      } else {
        int64_t pos = 0;
        for (int j = 0; j < k; ++j) pos += j == 0 ? T.Jm[0] * T.K : T.Jm[j];
        X = T.omega + pos;
      }
      TNR_TRY(prod_bwd(s, site_core(T, k), a, trans, X, S, Kx, S2, gIn[k], gAm[k], prev ? gX[k] : nullptr));
    }
    gOut = gX;
  }
  // merge adjoint: site 1 of A' back to A's leading cores
  {
    std::vector<int64_t> I0s(T.m), J0s(T.m);
    I0s[0] = T.A.I[0];
    J0s[0] = T.A.J[0];
    for (int j = 1; j < T.m; ++j) {
      I0s[j] = I0s[j - 1] * T.A.I[j];
      J0s[j] = J0s[j - 1] * T.A.J[j];
    }
    for (int j = 0; j < T.m; ++j)
      TNR_TRY(zero(s, dA->core[j], T.A.R[j] * T.A.I[j] * T.A.J[j] * T.A.R[j + 1]));
    double *g = gAm[0];
    for (int j = T.m - 1; j >= 1; --j) {
      const Site b{T.A.R[j], T.A.I[j], T.A.J[j], T.A.R[j + 1]};
      double *gPrev = j - 1 == 0 ? dA->core[0] : tmp.take(I0s[j - 1] * J0s[j - 1] * b.R);
      if (!gPrev) return TNR_ENOMEM;
      if (j - 1 > 0) TNR_TRY(zero(s, gPrev, I0s[j - 1] * J0s[j - 1] * b.R));
      TNR_TRY(merge_bwd(s, T.merged[j - 1], I0s[j - 1], J0s[j - 1], T.A.core[j], b, g, gPrev, dA->core[j]));
      g = gPrev;
    }
    if (T.m == 1) TNR_CK(cudaMemcpyAsync(dA->core[0], gAm[0], sizeof(double) * T.Im[0] * T.Jm[0] * T.RA[1],
                                         cudaMemcpyDeviceToDevice, s));
  }
  const int st = read_status(s);
  tmp.release();
  if (st != TNR_OK) return st;
  return tmp.ok ? TNR_OK : TNR_ENOMEM;
}

}  // namespace

extern "C" int tnr_diff_forward(const tnr_mpo *A, int32_t k, int32_t p, int32_t q, uint64_t seed, double *S,
                                void **tape, void *stream) {
  using namespace tnr;
  if (!A || !S || !tape || k < 1 || p < 0 || q < 0) return TNR_EINVAL;
  *tape = nullptr;
  if (A->d < 1 || A->d > TNR_MAX_SITES || A->R[0] != 1 || A->R[A->d] != 1) return TNR_EINVAL;
  if (A->dtype != TNR_F64 && A->dtype != TNR_F32) return TNR_EINVAL;
  for (int i = 0; i < A->d; ++i)
    if (A->I[i] < 1 || A->J[i] < 1 || A->R[i + 1] < 1 || !A->core[i]) return TNR_EINVAL;
  const int64_t K = (int64_t)k + p;
  int m = 0;
  {
    double pi = 1, pj = 1;
    for (int i = 0; i < A->d; ++i) {
      pi *= (double)A->I[i];
      pj *= (double)A->J[i];
      if (pi >= (double)K && pj >= (double)K) {
        m = i + 1;
        break;
      }
    }
  }
  if (m == 0) return TNR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DiffTape *T = new (std::nothrow) DiffTape();
  if (!T) return TNR_ENOMEM;
  T->mem.s = s;
  T->A = *A;
  if (A->dtype == TNR_F32) {  // the tape keeps float64 copies of the cores (exact widening)
    double *dst[TNR_MAX_SITES];
    for (int i = 0; i < A->d; ++i) {
      dst[i] = T->mem.take(A->R[i] * A->I[i] * A->J[i] * A->R[i + 1]);
      if (!dst[i]) {
        T->mem.release();
        delete T;
        return TNR_ENOMEM;
      }
    }
    const int rc = widen_cores(s, *A, dst, &T->A);
    if (rc != TNR_OK) {
      T->mem.release();
      cudaStreamSynchronize(s);
      delete T;
      return rc;
    }
  }
  T->m = m;
  T->d = A->d - m + 1;
  T->K = K;
  T->k = k;
  T->p = p;
  T->q = q;
  T->Im[0] = 1;
  T->Jm[0] = 1;
  for (int i = 0; i < m; ++i) {
    T->Im[0] *= A->I[i];
    T->Jm[0] *= A->J[i];
  }
  T->RA[0] = 1;
  for (int i = 1; i < T->d; ++i) {
    T->Im[i] = A->I[m - 1 + i];
    T->Jm[i] = A->J[m - 1 + i];
  }
  for (int i = 1; i <= T->d; ++i) T->RA[i] = A->R[m - 1 + i];
  const int rc = diff_forward(s, *T, seed, S);
  if (rc != TNR_OK) {
    T->mem.release();
    cudaStreamSynchronize(s);
    delete T;
    return rc;
  }
  *tape = T;
  return TNR_OK;
}

extern "C" int tnr_diff_backward(void *tape, const double *dS, tnr_mpo *dA, void *stream) {
  if (!tape || !dS || !dA) return TNR_EINVAL;
  DiffTape *T = static_cast<DiffTape *>(tape);
  if (dA->d != T->A.d || (dA->dtype != TNR_F64 && dA->dtype != TNR_F32)) return TNR_EINVAL;
  for (int i = 0; i < T->A.d; ++i)
    if (!dA->core[i]) return TNR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dA->dtype == TNR_F64) return diff_backward(s, *T, dS, dA);
  // float32 gradients: computed in float64 scratch, then rounded into the caller's cores
  tnr::Pool scratch;
  scratch.s = s;
  tnr_mpo g = *dA;
  g.dtype = TNR_F64;
  for (int i = 0; i < T->A.d; ++i) {
    g.core[i] = scratch.take(T->A.R[i] * T->A.I[i] * T->A.J[i] * T->A.R[i + 1]);
    if (!g.core[i]) {
      scratch.release();
      return TNR_ENOMEM;
    }
  }
  int rc = diff_backward(s, *T, dS, &g);
  for (int i = 0; i < T->A.d && rc == TNR_OK; ++i)
    rc = tnr::narrow_to_f32(s, g.core[i], reinterpret_cast<float *>(dA->core[i]),
                            T->A.R[i] * T->A.I[i] * T->A.J[i] * T->A.R[i + 1]);
  scratch.release();
  const cudaError_t e = cudaStreamSynchronize(s);
  return rc != TNR_OK ? rc : tnr::check_cuda(e);
}

extern "C" void tnr_diff_free(void *tape, void *stream) {
  if (!tape) return;
  DiffTape *T = static_cast<DiffTape *>(tape);
  T->mem.s = static_cast<cudaStream_t>(stream);
  T->mem.release();
  delete T;
}
