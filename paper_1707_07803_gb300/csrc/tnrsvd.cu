// TNrSVD on the GPU: MPO products (Section 5.2), MPO-QR with integrated rounding (Alg. 5.2,
// Section 5.4), MPO-SVD (Alg. 5.3) and the randomized MPO subspace iteration (Alg. 5.4).
//
// Host code orders the per-site steps (the sweeps are sequential over sites); every step
// runs in this library's kernels. Bond ranks chosen by the truncation are read back to the
// host after each bond so the next launch is sized exactly.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "dev_common.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

// ---------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------

// Per-site product, Section 5.2. Output core (R*S, Xo, Kx, R2*S2) with bonds r + R s.
//   trans = 0: Y((r,s), i, c, (r',s')) = sum_j A(r,i,j,r') X(s,j,c,s')
//   trans = 1: Y((r,s), j, c, (r',s')) = sum_i A(r,i,j,r') X(s,i,c,s')
// All sites of one product in a single launch (FP64): the threads of the grid stride over the
// concatenated outputs of the sites; site b owns outputs [off[b], off[b+1]).
struct ContractSite {
  const double *A, *X;
  double *Y;
  unsigned R, I, J, R2, S, Kx, S2;
};
struct ContractBatch {
  int n, trans;
  unsigned off[TNR_MAX_SITES + 1];
  ContractSite site[TNR_MAX_SITES];
};

__global__ void k_contract_sites(const __grid_constant__ ContractBatch B) {
  const unsigned total = B.off[B.n];
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int b = 0;
    while (idx >= B.off[b + 1]) ++b;
    const ContractSite &D = B.site[b];
    unsigned t = idx - B.off[b];
    const unsigned Xo = B.trans ? D.J : D.I, Ny = B.trans ? D.I : D.J;
    const unsigned RS = D.R * D.S;
    const unsigned rs = t % RS;
    t /= RS;
    const unsigned xo = t % Xo;
    t /= Xo;
    const unsigned c = t % D.Kx;
    const unsigned rs2 = t / D.Kx;
    const unsigned r = rs % D.R, s = rs / D.R;
    const unsigned r2 = rs2 % D.R2, s2 = rs2 / D.R2;
    const double *xp = D.X + s + (size_t)D.S * (Ny * (c + (size_t)D.Kx * s2));
    const double *ap = B.trans ? D.A + r + (size_t)D.R * (D.I * (xo + (size_t)D.J * r2))
                               : D.A + r + (size_t)D.R * (xo + D.I * ((size_t)D.J * r2));
    const unsigned as = B.trans ? D.R : D.R * D.I;
    double acc = 0.0;
    for (unsigned y = 0; y < Ny; ++y) acc = fma(ap[(size_t)as * y], xp[(size_t)D.S * y], acc);
    D.Y[idx - B.off[b]] = acc;
  }
}

// One step of the leading-site merge (Section 6.3): T (nr x nc x R) with core (R, I, J, R2)
// gives T' ((nr I) x (nc J) x R2), rows (a, i) -> a + nr i, columns (b, j) -> b + nc j.
__global__ void k_merge(const double *__restrict__ T, int64_t nr, int64_t nc, int64_t R, const double *__restrict__ C,
                        int64_t I, int64_t J, int64_t R2, double *__restrict__ out) {
  const unsigned NR = (unsigned)(nr * I), NC = (unsigned)(nc * J), total = NR * NC * (unsigned)R2;
  const unsigned unr = (unsigned)nr, unc = (unsigned)nc;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const unsigned row = idx % NR, col = (idx / NR) % NC, s = idx / (NR * NC);
    const unsigned a = row % unr, i = row / unr, b = col % unc, j = col / unc;
    double acc = 0.0;
    for (int64_t r = 0; r < R; ++r) acc = fma(T[a + nr * (b + nc * r)], C[r + R * (i + I * (j + J * s))], acc);
    out[idx] = acc;
  }
}

// Lemma 5.1 random MPO: SplitMix64 counter stream, uniforms ((z >> 11) + 1) 2^-53 in (0, 1],
// Box-Muller cosine branch, normal m from uniforms 2m and 2m+1.
__global__ void k_omega(uint64_t seed, int64_t count, double *out) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < count; m += (int64_t)gridDim.x * blockDim.x) {
    out[m] = omega_normal(seed, (uint64_t)m);
  }
}

// Site-1 permutation of Algs. 5.2/5.3: core (1, I1, K, t) <-> matrix A1^T of size (I1 t) x K,
// element (i + I1 r, c) <-> core (i, c, r). dir = 0: core -> matrix. dir = 1: matrix -> core,
// keeping only columns c < kout (core (1, I1, kout, t)).
__global__ void k_site1_perm(const double *__restrict__ src, double *__restrict__ dst, int64_t I1, int64_t K,
                             int64_t t, int64_t kout, int dir) {
  const unsigned total = (unsigned)(dir == 0 ? I1 * K * t : I1 * kout * t);
  const unsigned kk = (unsigned)(dir == 0 ? K : kout), uI1 = (unsigned)I1;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const unsigned i = idx % uI1, c = (idx / uI1) % kk, r = idx / (uI1 * kk);
    const size_t mi = (i + (size_t)I1 * r) + (size_t)(I1 * t) * c;
    if (dir == 0)
      dst[mi] = src[idx];
    else
      dst[idx] = src[mi];
  }
}

__global__ void k_widen(const float *__restrict__ x, double *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void k_narrow(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void __launch_bounds__(1024) k_norm2(const double *__restrict__ x, int64_t n, double *out, int *status) {
  __shared__ double red[32];
  double s = 0.0;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < n; i += 1024) {
    const double v = x[i];
    if (!isfinite(v)) bad = true;
    s = fma(v, v, s);
  }
  if (bad) set_status(status, TNR_ENONFINITE);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t += red[w];
    *out = t;
  }
}

// Truncation rule: delta^2 = tol^2 ||Y||^2 / (d - 1); keep the smallest r >= 1 with
// sum_{l >= r} s_l^2 <= delta^2, then r <= max_rank.
__global__ void k_trunc(const double *__restrict__ S, int64_t n, const double *norm2, double tol, int64_t dm1,
                        int64_t max_rank, int64_t *r_out, int *status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double delta2 = dm1 > 0 ? tol * tol * (*norm2) / (double)dm1 : 0.0;
  double tail = 0.0;
  int64_t r = n;
  // tail(r) = sum_{l >= r} s_l^2, computed from the back (same order as the definition)
  for (int64_t cand = n - 1; cand >= 1; --cand) {
    tail += S[cand] * S[cand];
    if (tail <= delta2)
      r = cand;
    else
      break;
  }
  for (int64_t l = 0; l < n; ++l)
    if (!isfinite(S[l])) set_status(status, TNR_ENONFINITE);
  if (max_rank > 0 && r > max_rank) r = max_rank;
  if (r < 1) r = 1;
  *r_out = r;
}

int grid_for(int64_t work, int threads = 256) {
  int64_t g = cdiv(work, threads);
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------------------------------
// Host-side MPO helpers
// ---------------------------------------------------------------------------------------
int64_t core_elems(const tnr_mpo &M, int k) { return M.R[k] * M.I[k] * M.J[k] * M.R[k + 1]; }

}  // namespace

int validate_input(const tnr_mpo *A, bool allow_f32) {
  if (!A || A->d < 1 || A->d > TNR_MAX_SITES) return TNR_EINVAL;
  if (A->dtype != TNR_F64 && !(allow_f32 && A->dtype == TNR_F32)) return TNR_EINVAL;
  if (A->R[0] != 1 || A->R[A->d] != 1) return TNR_EINVAL;
  for (int k = 0; k < A->d; ++k) {
    if (A->I[k] < 1 || A->J[k] < 1 || A->R[k + 1] < 1 || !A->core[k]) return TNR_EINVAL;
  }
  return TNR_OK;
}

namespace {

struct Bufs {
  double *tmp = nullptr;    // GEMM / copy staging, max core
  double *Rbuf = nullptr;   // R factors
  double *Mq = nullptr;     // matrix copies for QR-of-SVD
  double *Rm = nullptr;     // small square factors
  double *G = nullptr;      // Jacobi input/U
  double *Vr = nullptr;     // Jacobi V
  double *Sv = nullptr;     // singular values
  double *US = nullptr;     // U * S
  void *qr = nullptr;       // QR scratch
  void *jac = nullptr;      // Jacobi scratch
  double *norm2 = nullptr;  // device scalar
  int64_t *rdev = nullptr;  // device ranks: 2 x (TNR_MAX_SITES + 1) (compression, then rounding)
  unsigned *bar = nullptr;  // grid-barrier state of the cooperative compression
  int *ctl = nullptr;       // its control word
  int64_t cap = 0;          // doubles in tmp, Mq and US
};

void carve(Arena &ar, const Limits &L, Bufs &b) {
  b.tmp = ar.take<double>(L.maxcore);
  b.Rbuf = ar.take<double>(L.maxbond * L.maxbond);
  b.Mq = ar.take<double>(L.maxcore);
  b.Rm = ar.take<double>(L.maxsq * L.maxsq);
  b.G = ar.take<double>(L.maxsq * L.maxsq);
  b.Vr = ar.take<double>(L.maxsq * L.maxsq);
  b.Sv = ar.take<double>(L.maxsq);
  b.US = ar.take<double>(L.maxcore);
  // every QR factors a core-sized matrix (m * n <= maxcore) with n <= max(maxbond, maxsq)
  b.qr = ar.take<char>(std::max(qr_scratch_bound(L.maxcore, std::max(L.maxbond, L.maxsq)),
                                 qrcp_scratch_bound(L.maxcore, std::max(L.maxbond, L.maxsq))));
  b.jac = ar.take<char>(std::max<size_t>(jacobi_scratch(L.maxsq), 256));
  b.norm2 = ar.take<double>(1);
  b.rdev = ar.take<int64_t>(2 * (TNR_MAX_SITES + 1));  // compression ranks, then rounded ranks
  b.bar = ar.take<unsigned>(4);
  b.ctl = ar.take<int>(4);
  b.cap = L.maxcore;
}

int d2h_rank(cudaStream_t s, const int64_t *rdev, int64_t *r) {
  const ReadBack rb[1] = {{r, rdev, sizeof(int64_t)}};
  int st = read_back(s, rb, 1);
  return st;
}

// Exact right-to-left compression before the rounding sweeps (used when tol > 0). Products
// multiply ranks (R_k S_k) but their numerical ranks are often far lower, and the redundancy
// sits in the right parts of the product (e.g. A^T Q = V (S U^T Q) keeps V's bonds), where a
// left-to-right orthogonalisation cannot see it. For k = d-1..1: M_k (t x w) = L Q_k by a
// column-pivoted QR of M_k^T that stops once every remaining column norm is below
// cut * ||M_k||_F (see compress_cut); Q_k (orthonormal rows) replaces the core and L
// is absorbed into core k-1. Only directions at the rounding level of M_k are dropped (the size
// of a Householder factorisation's own backward error, far below the truncation threshold), so
// the rounding that follows returns the same result to rounding accuracy, on bonds of the
// numerical rank instead of R_k S_k. Every compressed core Q_k has orthonormal rows, so when all
// bonds were compressed (*all_bonds) cores 1..d-1 leave right-orthonormal.
int compress_rl(cudaStream_t s, tnr_mpo &Y, Bufs &b, double cut, bool *all_bonds, int start) {
  *all_bonds = true;
  for (int k = start; k >= 1; --k) {
    const int64_t t = Y.R[k], w = Y.I[k] * Y.J[k] * Y.R[k + 1];
    int64_t r = 0;
    if (qr_small_fits(w, t)) {
      // M^T (w x t) = Q~ R~ P^T; core_k <- Q~^T (r x w, packed), b.Rbuf <- R~^T (t x r)
      TNR_TRY(qr_small_f64(s, Y.core[k], t, w, t, true, true, cut, Y.core[k], 0, true, b.Rbuf, t, true, b.rdev));
      TNR_TRY(d2h_rank(s, b.rdev, &r));
      {  // r Householder steps on the w x t matrix, plus the explicit w x r Q
        const double M = (double)w, N = (double)t, rr = (double)r;
        stats_work(K_QR_PIV, 4 * M * N * rr - 2 * (M + N) * rr * rr + 4 * rr * rr * rr / 3 + 2 * M * rr * rr -
                                 2 * rr * rr * rr / 3);
      }
    } else {
      TNR_TRY(copy_matrix_f64(s, Y.core[k], t, b.Mq, w, w, t, true));  // M^T (w x t)
      bool used = false;
      TNR_TRY(qrcp_f64(s, b.Mq, w, t, w, b.US, std::min(w, t), cut, b.qr, b.rdev, &used));
      if (!used) {  // too large for the pivoted kernels: leave this bond as it is
        *all_bonds = false;
        continue;
      }
      TNR_TRY(d2h_rank(s, b.rdev, &r));
      TNR_TRY(copy_matrix_f64(s, b.Mq, w, Y.core[k], r, r, w, true));   // Q~^T (r x w)
      TNR_TRY(copy_matrix_f64(s, b.US, std::min(w, t), b.Rbuf, t, t, r, true));  // R~^T (t x r)
    }
    const int64_t rows = Y.R[k - 1] * Y.I[k - 1] * Y.J[k - 1];
    TNR_TRY(gemm_f64(s, false, false, rows, r, t, 1.0, Y.core[k - 1], rows, 0, b.Rbuf, t, 0, 0.0, b.tmp, rows, 0));
    TNR_CK(cudaMemcpyAsync(Y.core[k - 1], b.tmp, sizeof(double) * rows * r, cudaMemcpyDeviceToDevice, s));
    Y.R[k] = r;
  }
  return TNR_OK;
}


// Left-to-right Householder QR sweep (rounding part 1, Section 5.4): core k reshaped
// (R_k I_k J_k) x R_{k+1} = Q R; Q replaces the core, R is absorbed into core k+1.
int sweep_lr(cudaStream_t s, tnr_mpo &Y, Bufs &b) {
  for (int k = 0; k + 1 < Y.d; ++k) {
    const int64_t rows = Y.R[k] * Y.I[k] * Y.J[k], cols = Y.R[k + 1];
    const int64_t n = std::min(rows, cols);
    if (qr_small_fits(rows, cols))
      TNR_TRY(qr_small_f64(s, Y.core[k], rows, rows, cols, false, false, 0.0, Y.core[k], rows, false, b.Rbuf, n, false,
                           nullptr));
    else
      TNR_TRY(qr_f64(s, Y.core[k], rows, cols, rows, b.Rbuf, n, b.qr));
    const int64_t w = Y.I[k + 1] * Y.J[k + 1] * Y.R[k + 2];
    TNR_TRY(gemm_f64(s, false, false, n, w, cols, 1.0, b.Rbuf, n, 0, Y.core[k + 1], cols, 0, 0.0, b.tmp, n, 0));
    TNR_CK(cudaMemcpyAsync(Y.core[k + 1], b.tmp, sizeof(double) * n * w, cudaMemcpyDeviceToDevice, s));
    Y.R[k + 1] = n;
  }
  return TNR_OK;
}

// Plain thin QR: A (m x n, lda = m) <- Q, R (min x n, ldr). Matrices with many long columns
// (m >= 128, n >= 16) go to the multi-CTA kernel, whose FP64 work spreads over n SMs; the
// rest to the one-CTA shared-memory kernel.
int thin_qr(cudaStream_t s, double *A, int64_t m, int64_t n, double *R, int64_t ldr, Bufs &b) {
  if (qr_small_fits(m, n) && !(m >= 128 && n >= 16))
    return qr_small_f64(s, A, m, m, n, false, false, 0.0, A, m, false, R, ldr, false, nullptr);
  return qr_f64(s, A, m, n, m, R, ldr, b.qr);
}

// Truncated SVD of M (t x w, ld t) for the right-to-left sweep: writes V^T[:r] (r x w) into
// `core_out`, U[:, :r] diag(S[:r]) (t x r, ld t) into b.US, returns r.
int svd_trunc(cudaStream_t s, const double *M, int64_t t, int64_t w, double tol, int64_t dm1, int64_t max_rank,
              double *core_out, Bufs &b, int64_t *r_out) {
  int64_t r = 0;
  if (t >= w) {
    TNR_TRY(copy_matrix_f64(s, M, t, b.Mq, t, t, w, false));
    TNR_TRY(thin_qr(s, b.Mq, t, w, b.Rm, w, b));  // Mq <- Q_m (t x w), Rm (w x w)
    TNR_TRY(jacobi_svd_f64(s, b.Rm, w, w, b.Sv, b.Vr, w, b.jac));  // Rm <- U_r
    {
      LaunchScope ls(K_MISC, s);
      k_trunc<<<1, 32, 0, s>>>(b.Sv, w, b.norm2, tol, dm1, max_rank, b.rdev, status_ptr());
    }
    TNR_TRY(d2h_rank(s, b.rdev, &r));
    TNR_TRY(copy_matrix_f64(s, b.Vr, w, core_out, r, r, w, true));  // V_r[:, :r]^T
    TNR_TRY(scale_columns_f64(s, b.Rm, w, w, r, b.Sv));
    TNR_TRY(gemm_f64(s, false, false, t, r, w, 1.0, b.Mq, t, 0, b.Rm, w, 0, 0.0, b.US, t, 0));
  } else {
    TNR_TRY(copy_matrix_f64(s, M, t, b.Mq, w, w, t, true));  // M^T (w x t)
    TNR_TRY(thin_qr(s, b.Mq, w, t, b.Rm, t, b));  // Mq <- Q_m (w x t), Rm (t x t)
    TNR_TRY(copy_matrix_f64(s, b.Rm, t, b.G, t, t, t, true));  // G = Rm^T
    TNR_TRY(jacobi_svd_f64(s, b.G, t, t, b.Sv, b.Vr, t, b.jac));  // G <- U
    {
      LaunchScope ls(K_MISC, s);
      k_trunc<<<1, 32, 0, s>>>(b.Sv, t, b.norm2, tol, dm1, max_rank, b.rdev, status_ptr());
    }
    TNR_TRY(d2h_rank(s, b.rdev, &r));
    // V^T[:r] = V_r[:, :r]^T Q_m^T  (r x w)
    TNR_TRY(gemm_f64(s, true, true, r, w, t, 1.0, b.Vr, t, 0, b.Mq, w, 0, 0.0, core_out, r, 0));
    TNR_TRY(scale_columns_f64(s, b.G, t, t, r, b.Sv));
    TNR_TRY(copy_matrix_f64(s, b.G, t, b.US, t, t, r, false));
  }
  *r_out = r;
  return TNR_OK;
}

// Right-to-left truncating sweep (rounding part 2 fused with the loop of Alg. 5.2).
int sweep_rl(cudaStream_t s, tnr_mpo &Y, double tol, int64_t max_rank, Bufs &b) {
  if (Y.d < 2) return TNR_OK;
  {
    LaunchScope ls(K_MISC, s);
    k_norm2<<<1, 1024, 0, s>>>(Y.core[Y.d - 1], core_elems(Y, Y.d - 1), b.norm2, status_ptr());
  }
  TNR_CK(cudaGetLastError());
  for (int k = Y.d - 1; k >= 1; --k) {
    const int64_t t = Y.R[k], w = Y.I[k] * Y.J[k] * Y.R[k + 1];
    int64_t r = 0;
    if (svd_step_smem(t, w) <= 200 * 1024 && std::min(t, w) <= 1024) {
      // one fused launch: QR of the narrow side, Jacobi SVD, truncation, V^T rows and U S
      TNR_TRY(svd_step_small(s, Y.core[k], t, w, b.norm2, tol, Y.d - 1, max_rank, Y.core[k], b.US, b.rdev));
      TNR_TRY(d2h_rank(s, b.rdev, &r));
    } else {
      TNR_TRY(svd_trunc(s, Y.core[k], t, w, tol, Y.d - 1, max_rank, b.tmp, b, &r));
      TNR_CK(cudaMemcpyAsync(Y.core[k], b.tmp, sizeof(double) * r * w, cudaMemcpyDeviceToDevice, s));
    }
    const int64_t rows = Y.R[k - 1] * Y.I[k - 1] * Y.J[k - 1];
    TNR_TRY(gemm_f64(s, false, false, rows, r, t, 1.0, Y.core[k - 1], rows, 0, b.US, t, 0, 0.0, b.tmp, rows, 0));
    TNR_CK(cudaMemcpyAsync(Y.core[k - 1], b.tmp, sizeof(double) * rows * r, cudaMemcpyDeviceToDevice, s));
    Y.R[k] = r;
  }
  return TNR_OK;
}

// Both rounding sweeps of Section 5.4 (L->R QR, then the R->L truncating loop of Alg. 5.2): one
// fused one-CTA launch when every core fits shared memory, else one launch sequence per bond.
// right_orth: cores 1..d-1 are right-orthonormal on entry (see compress_rl).
// *pending: the fused kernel ran and left the ranks in b.rdev (Y.R keeps the bounds it had on
// entry until read_ranks); otherwise Y.R is exact on return.
int round_sweeps(cudaStream_t s, tnr_mpo &Y, double tol, int64_t max_rank, bool right_orth, Bufs &b, bool *pending) {
  *pending = false;
  bool fused = false;
  TNR_TRY(round_small(s, Y, tol, max_rank, right_orth, b.rdev, &fused));
  if (!fused) {
    TNR_TRY(sweep_lr(s, Y, b));
    return sweep_rl(s, Y, tol, max_rank, b);
  }
  *pending = true;
  return TNR_OK;
}

// Reads the ranks the fused rounding left in b.rdev and the site-1 fallback flag (one sync).
int read_ranks(cudaStream_t s, tnr_mpo &Y, Bufs &b, bool pending, int *hflag) {
  int64_t R[TNR_MAX_SITES + 1];
  const ReadBack rb[2] = {{hflag, b.ctl + 1, sizeof(int)}, {R, b.rdev, sizeof(int64_t) * (Y.d + 1)}};
  TNR_TRY(read_back(s, rb, pending ? 2 : 1));
  if (pending)
    for (int k = 0; k <= Y.d; ++k) Y.R[k] = R[k];
  return TNR_OK;
}

int site1_perm(cudaStream_t s, const double *src, double *dst, int64_t I1, int64_t K, int64_t t, int64_t kout,
               int dir) {
  LaunchScope ls(K_MISC, s);
  k_site1_perm<<<grid_for(I1 * K * t), 256, 0, s>>>(src, dst, I1, K, t, kout, dir);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// Thin QR of the site-1 matrix A1^T = Q~ R~ ((I1 t) x K, Alg. 5.2/5.3), R~ into b.Rm, Q~ into b.Mq
// (column-major) or, with core_out, back into the site-1 core. For K <= 32: CholeskyQR2 in one
// cooperative launch (site1_qr.cu) that reads the rank left by the fused rounding on the device
// when `pending`; the ranks and its fallback flag come back in one sync. When a Cholesky breaks
// down or the second pass is not near the identity (cond(A1) beyond ~1e8) the QR is redone by the
// multi-CTA Householder kernel on the unchanged core.
// Householder QR of the site-1 matrix (the CholeskyQR2 fallback), Y.R exact.
int site1_householder(cudaStream_t s, tnr_mpo &Y, bool core_out, Bufs &b) {
  const int64_t I1 = Y.I[0], K = Y.J[0], t = Y.R[1];
  if (I1 * t < K) return TNR_EINVAL;
  TNR_TRY(site1_perm(s, Y.core[0], b.Mq, I1, K, t, K, 0));
  TNR_TRY(thin_qr(s, b.Mq, I1 * t, K, b.Rm, K, b));
  if (core_out) TNR_TRY(site1_perm(s, b.Mq, Y.core[0], I1, K, t, K, 1));
  return TNR_OK;
}

int site1_qr(cudaStream_t s, tnr_mpo &Y, bool pending, bool core_out, Bufs &b) {
  const int64_t I1 = Y.I[0], K = Y.J[0];
  bool launched = false;
  int *flag = b.ctl + 1;
  TNR_TRY(site1_cholqr2(s, Y.core[0], I1, K, Y.R[1], pending ? b.rdev + 1 : nullptr, core_out, nullptr, b.US, b.cap,
                        b.Vr, b.Rm, b.Mq, flag, b.bar, &launched));
  int hflag = 1;
  if (launched) {
    TNR_TRY(read_ranks(s, Y, b, pending, &hflag));
  } else if (pending) {
    int dummy = 0;
    TNR_TRY(read_ranks(s, Y, b, true, &dummy));
  }
  if (I1 * Y.R[1] < K) return TNR_EINVAL;
  if (!hflag) return TNR_OK;
  return site1_householder(s, Y, core_out, b);
}

// Compression, rounding and the site-1 QR of a product MPO (Section 5.4 and the site-1 step of
// Algs. 5.2/5.3) with one host round trip when the shapes allow: the cooperative compression runs
// the rounding sweeps at its end (fused), the CholeskyQR2 of the site-1 matrix follows at once
// (reading the rounded rank on the device, run only if the rounding ran), and the ranks, the
// control words and the QR's fallback flag come back together. Whatever a fused stage declined
// (a bond too wide for the one-CTA QR, cores beyond the rounding's shared memory, a CholeskyQR2
// that must be redone) continues on the host-driven path from that point.
int reduce_and_site1(cudaStream_t s, tnr_mpo &Y, double tol, int64_t max_rank, double cut, bool core_out, Bufs &b) {
  bool right_orth = false, pending = false;
  if (tol > 0.0 && Y.d >= 2) {
    bool launched = false;
    int64_t *Rround = b.rdev + (TNR_MAX_SITES + 1);
    TNR_TRY(compress_launch(s, Y, cut, b.Rbuf, b.tmp, b.Mq, b.cap, b.bar, b.ctl, b.rdev, true, tol, max_rank,
                            Rround, &launched));
    if (launched) {
      bool s1 = false;
      TNR_TRY(site1_cholqr2(s, Y.core[0], Y.I[0], Y.J[0], Y.R[1], Rround + 1, core_out, b.ctl + 2, b.US, b.cap, b.Vr,
                            b.Rm, b.Mq, b.ctl + 1, b.bar, &s1));
      int64_t h[2 * (TNR_MAX_SITES + 1)];
      int hctl[3] = {0, 0, 0};
      const ReadBack rb[2] = {{h, b.rdev, sizeof(int64_t) * 2 * (TNR_MAX_SITES + 1)}, {hctl, b.ctl, sizeof(hctl)}};
      TNR_TRY(read_back(s, rb, 2));
      const int next = hctl[0];
      compress_record_work(Y, h, next);
      for (int k = next + 1; k < Y.d; ++k) Y.R[k] = h[k];
      if (next != 0) {  // a bond too wide for the one-CTA QR: the host-driven sweep continues
        TNR_TRY(compress_rl(s, Y, b, cut, &right_orth, next));
        TNR_TRY(round_sweeps(s, Y, tol, max_rank, right_orth, b, &pending));
        return site1_qr(s, Y, pending, core_out, b);
      }
      if (hctl[2] == 0) {  // compressed cores beyond the fused rounding's shared memory
        TNR_TRY(round_sweeps(s, Y, tol, max_rank, true, b, &pending));
        return site1_qr(s, Y, pending, core_out, b);
      }
      const int64_t *hr = h + (TNR_MAX_SITES + 1);
      for (int k = 0; k <= Y.d; ++k) Y.R[k] = hr[k];
      if (Y.I[0] * Y.R[1] < Y.J[0]) return TNR_EINVAL;
      if (!s1) return site1_qr(s, Y, false, core_out, b);
      if (hctl[1]) return site1_householder(s, Y, core_out, b);
      return TNR_OK;
    }
    TNR_TRY(compress_rl(s, Y, b, cut, &right_orth, Y.d - 1));
  }
  TNR_TRY(round_sweeps(s, Y, tol, max_rank, right_orth, b, &pending));
  if (Y.I[0] * Y.R[1] < Y.J[0] && !pending) return TNR_EINVAL;
  return site1_qr(s, Y, pending, core_out, b);
}

// MPO-QR with integrated rounding (Alg. 5.2 + Section 5.4). Y is a tall matrix MPO with K
// columns on site 1 (Y.J[0] = K, Y.J[k>0] = 1). Rout (K x K) may be null.
int orthogonalize_impl(cudaStream_t s, tnr_mpo &Y, double *Rout, double tol, int64_t max_rank, Bufs &b,
                       bool mixed_product = false) {
  // A1^T = Q~ R~ with Q~ back into the site-1 core
  TNR_TRY(reduce_and_site1(s, Y, tol, max_rank, compress_cut(tol, mixed_product), true, b));
  if (Rout) TNR_CK(cudaMemcpyAsync(Rout, b.Rm, sizeof(double) * Y.J[0] * Y.J[0], cudaMemcpyDeviceToDevice, s));
  return TNR_OK;
}

// MPO-SVD (Alg. 5.3 + Section 5.4) of B = Z^T, Z a tall matrix MPO (rows J, K columns on
// site 1). Writes W (K x K) into Wout, S (K) into Sout, and V^(1) restricted to the first
// kout columns into V1 (core (1, J1, kout, t2)). Z's other cores become V's cores.
int mpo_svd_impl(cudaStream_t s, tnr_mpo &Z, double tol, int64_t max_rank, Bufs &b, double *Wout, double *Sout,
                 double *V1, int64_t kout, int64_t v1cap) {
  TNR_TRY(reduce_and_site1(s, Z, tol, max_rank, compress_cut(tol, false), false, b));  // M^T = Q~ R~
  const int64_t J1 = Z.I[0], K = Z.J[0], t = Z.R[1];
  const int64_t m = J1 * t;
  if (J1 * kout * t > v1cap) return TNR_ENOMEM;
  TNR_TRY(copy_matrix_f64(s, b.Rm, K, Wout, K, K, K, true));  // R~^T
  TNR_TRY(jacobi_svd_f64(s, Wout, K, K, Sout, b.Vr, K, b.jac));  // R~^T = W S Zr^T
  // V = Q~ Zr ((J1 t) x K), then V^(1) columns < kout
  TNR_TRY(gemm_f64(s, false, false, m, K, K, 1.0, b.Mq, m, 0, b.Vr, K, 0, 0.0, b.US, m, 0));
  TNR_TRY(site1_perm(s, b.US, V1, J1, K, t, kout, 1));
  return TNR_OK;
}

// Y = op(A) X (Section 5.2). The dense site-1 product goes to the tensor cores in mixed mode; every
// other site runs in FP64 in one launch for the whole product (an FP32 or BF16 product of FP64
// operands on CUDA cores would spend more FP64-pipe slots on conversions than the FP64 FMAs).
int contract_impl(cudaStream_t s, const tnr_mpo &A, int trans, const tnr_mpo &X, tnr_mpo &Y, bool mixed = false) {
  Y.d = A.d;
  Y.R[0] = 1;
  ContractBatch B;
  B.n = 0;
  B.trans = trans;
  B.off[0] = 0;
  double work = 0.0;
  for (int k = 0; k < A.d; ++k) {
    const int64_t R = A.R[k], I = A.I[k], J = A.J[k], R2 = A.R[k + 1];
    const int64_t S = X.R[k], Kx = X.J[k], S2 = X.R[k + 1];
    const int64_t Xo = trans ? J : I;
    const int64_t Ny = trans ? I : J;
    if (X.I[k] != Ny) return TNR_EINVAL;
    const int64_t total = R * S * Xo * Kx * R2 * S2;
    if (total > Y.cap[k]) return TNR_ENOMEM;
    Y.I[k] = Xo;
    Y.J[k] = Kx;
    Y.R[k + 1] = R2 * S2;
    if (mixed && R == 1 && S == 1 && Ny >= 16) {
      // dense site product on the tensor cores (BF16 x3 split, FP32 accumulation)
      TNR_TRY(contract_site1_tc(s, A.core[k], I, J, R2, X.core[k], Kx, S2, trans, Y.core[k], true));
      continue;
    }
    if ((double)B.off[B.n] + (double)total >= 4294967295.0) return TNR_ERANGE;
    ContractSite &D = B.site[B.n];
    D.A = A.core[k];
    D.X = X.core[k];
    D.Y = Y.core[k];
    D.R = (unsigned)R;
    D.I = (unsigned)I;
    D.J = (unsigned)J;
    D.R2 = (unsigned)R2;
    D.S = (unsigned)S;
    D.Kx = (unsigned)Kx;
    D.S2 = (unsigned)S2;
    B.off[B.n + 1] = B.off[B.n] + (unsigned)total;
    ++B.n;
    work += 2.0 * (double)total * (double)Ny;
  }
  if (B.n == 0 || B.off[B.n] == 0) return TNR_OK;
  stats_work(K_CONTRACT, work);
  LaunchScope ls(K_CONTRACT, s);
  k_contract_sites<<<grid_for(B.off[B.n]), 256, 0, s>>>(B);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

// Structural bound of bond b (1..d-1) of a (prod dims) x K matrix MPO with K on site 1.
int64_t tall_bound(const int64_t *dims, int d, int64_t K, int b) {
  double left = (double)K, right = 1.0;
  for (int i = 0; i < b; ++i) left *= (double)dims[i];
  for (int i = b; i < d; ++i) right *= (double)dims[i];
  double v = std::min(left, right);
  return v > 4e18 ? (int64_t)4e18 : (int64_t)v;
}


}  // namespace

int make_plan(const tnr_mpo *A, int64_t K, const tnr_opts *o, Plan &P) {
  TNR_TRY(validate_input(A, true));
  if (K < 1) return TNR_EINVAL;
  if (o && o->rounding != TNR_ROUND_TWO_SWEEP && o->rounding != TNR_ROUND_ZIPUP) return TNR_EINVAL;
  const bool zip = o && o->rounding == TNR_ROUND_ZIPUP;
  double pi = 1, pj = 1;
  int m = 0;
  for (int k = 0; k < A->d; ++k) {
    pi *= (double)A->I[k];
    pj *= (double)A->J[k];
    if (pi >= (double)K && pj >= (double)K) {
      m = k + 1;
      break;
    }
  }
  if (m == 0) return TNR_EINVAL;
  P.m = m;
  P.d = A->d - m + 1;
  P.I[0] = 1;
  P.J[0] = 1;
  for (int k = 0; k < m; ++k) {
    P.I[0] *= A->I[k];
    P.J[0] *= A->J[k];
  }
  P.RA[0] = 1;
  P.RA[1] = A->R[m];
  for (int k = 1; k < P.d; ++k) {
    P.I[k] = A->I[m - 1 + k];
    P.J[k] = A->J[m - 1 + k];
    P.RA[k + 1] = A->R[m + k];
  }
  const int64_t maxr = o ? o->max_rank : 0;
  P.sq[0] = 1;
  P.sq[P.d] = 1;
  for (int b = 1; b < P.d; ++b) {
    int64_t v = std::max(tall_bound(P.I, P.d, K, b), tall_bound(P.J, P.d, K, b));
    if (maxr > 0) v = std::min(v, maxr);
    P.sq[b] = v;
  }
  P.L = Limits();
  for (int k = 0; k < P.d; ++k) {
    const int64_t X = std::max(P.I[k], P.J[k]);
    const int64_t Kx = k == 0 ? K : 1;
    const int64_t b0 = P.RA[k] * P.sq[k], b1 = P.RA[k + 1] * P.sq[k + 1];
    const double cap = (double)b0 * (double)X * (double)Kx * (double)b1;
    // product core over 16 GB: outside the supported sizes (a zip-up rounding never forms it)
    if (cap > 2e9 && !zip) return TNR_ENOMEM;
    P.pcap[k] = (int64_t)cap;
    P.L.maxcore = std::max(P.L.maxcore, P.pcap[k]);
    P.L.maxbond = std::max(P.L.maxbond, std::max(b0, b1));
    P.L.maxrows = std::max(P.L.maxrows, b0 * X * Kx);
  }
  // square factors: min(t, w) of the R->L SVDs and K of the site-1 step
  P.L.maxsq = std::max<int64_t>(K, 1);
  for (int k = 1; k < P.d; ++k) {
    const int64_t X = std::max(P.I[k], P.J[k]);
    const int64_t t = P.RA[k] * P.sq[k], w = X * P.RA[k + 1] * P.sq[k + 1];
    P.L.maxsq = std::max(P.L.maxsq, std::min(t, w));
  }
  P.L.maxcore = std::max(P.L.maxcore, std::max(P.I[0], P.J[0]) * K * P.L.maxbond);
  if (P.L.maxsq > 1024 && !zip) return TNR_ENOMEM;  // Jacobi kernel limit (zip-up: checked per plan)
  P.omega_len = P.J[0] * K;
  for (int k = 1; k < P.d; ++k) P.omega_len += P.J[k];
  P.merged_elems = 0;
  if (m > 1) {
    int64_t nr = A->I[0], nc = A->J[0];
    for (int k = 1; k < m; ++k) {
      nr *= A->I[k];
      nc *= A->J[k];
      P.merged_elems = std::max(P.merged_elems, nr * nc * A->R[k + 1]);
    }
  }
  return TNR_OK;
}

int64_t mpo_elems(const tnr_mpo &A) {
  int64_t n = 0;
  for (int k = 0; k < A.d; ++k) n += A.R[k] * A.I[k] * A.J[k] * A.R[k + 1];
  return n;
}

int widen_cores(cudaStream_t s, const tnr_mpo &A, double *const *dst, tnr_mpo *out) {
  *out = A;
  out->dtype = TNR_F64;
  for (int k = 0; k < A.d; ++k) {
    const int64_t n = A.R[k] * A.I[k] * A.J[k] * A.R[k + 1];
    {
      LaunchScope ls(K_MISC, s);
      k_widen<<<grid_for(n), 256, 0, s>>>(reinterpret_cast<const float *>(A.core[k]), dst[k], n);
    }
    TNR_CK(cudaGetLastError());
    out->core[k] = dst[k];
  }
  return TNR_OK;
}

int narrow_to_f32(cudaStream_t s, const double *x, float *y, int64_t n) {
  if (n <= 0) return TNR_OK;
  LaunchScope ls(K_MISC, s);
  k_narrow<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

namespace {

struct SolveBufs {
  double *widened[TNR_MAX_SITES] = {nullptr};  // float64 copies of TNR_F32 input cores
  double *merged = nullptr, *merge_tmp = nullptr;
  double *omega = nullptr;
  double *P0[TNR_MAX_SITES], *P1[TNR_MAX_SITES];
  double *W = nullptr, *S = nullptr;
  Bufs b;
};

void carve_solve(Arena &ar, const Plan &P, int64_t K, SolveBufs &sb, const tnr_mpo *A) {
  if (A->dtype == TNR_F32)
    for (int k = 0; k < A->d; ++k) sb.widened[k] = ar.take<double>(A->R[k] * A->I[k] * A->J[k] * A->R[k + 1]);
  if (P.m > 1) {
    sb.merged = ar.take<double>(P.merged_elems);
    sb.merge_tmp = ar.take<double>(P.merged_elems);
  }
  sb.omega = ar.take<double>(P.omega_len);
  for (int k = 0; k < P.d; ++k) sb.P0[k] = ar.take<double>(P.pcap[k]);
  for (int k = 0; k < P.d; ++k) sb.P1[k] = ar.take<double>(P.pcap[k]);
  sb.W = ar.take<double>(K * K);
  sb.S = ar.take<double>(K);
  carve(ar, P.L, sb.b);
}

int merge_leading(cudaStream_t s, const tnr_mpo *A, const Plan &P, SolveBufs &sb, double **out) {
  if (P.m == 1) {
    *out = A->core[0];
    return TNR_OK;
  }
  // T starts as core 1 (I1 x J1 x R2); ping-pong so the last step lands in sb.merged.
  const double *T = A->core[0];
  int64_t nr = A->I[0], nc = A->J[0], R = A->R[1];
  for (int k = 1; k < P.m; ++k) {
    double *dst = ((P.m - 1 - k) % 2 == 0) ? sb.merged : sb.merge_tmp;
    const int64_t total = nr * A->I[k] * nc * A->J[k] * A->R[k + 1];
    {
      LaunchScope ls(K_MERGE, s);
      k_merge<<<grid_for(total), 256, 0, s>>>(T, nr, nc, R, A->core[k], A->I[k], A->J[k], A->R[k + 1], dst);
    }
    TNR_CK(cudaGetLastError());
    T = dst;
    nr *= A->I[k];
    nc *= A->J[k];
    R = A->R[k + 1];
  }
  *out = sb.merged;
  return TNR_OK;
}

int solve_impl(cudaStream_t s, const tnr_mpo *A, int32_t k, int32_t p, int32_t q, uint64_t seed, const tnr_opts *o,
               tnr_mpo *U, double *S, tnr_mpo *V, void *ws, size_t ws_bytes) {
  if (k < 1 || p < 0 || q < 0 || !U || !V || !S || !o) return TNR_EINVAL;
  if (o->precision != TNR_FP64 && o->precision != TNR_MIXED) return TNR_EINVAL;
  if (o->rounding != TNR_ROUND_TWO_SWEEP) return TNR_EINVAL;  // zip-up: persistent batch only
  const int64_t K = (int64_t)k + p;
  Plan P;
  TNR_TRY(make_plan(A, K, o, P));
  Arena ar;
  ar.base = static_cast<char *>(ws);
  ar.size = ws_bytes;
  SolveBufs sb;
  carve_solve(ar, P, K, sb, A);
  if (!ar.ok || !ws) return TNR_ENOMEM;
  // output capacities
  if (U->d != P.d || V->d != P.d || U->dtype != TNR_F64 || V->dtype != TNR_F64) return TNR_EINVAL;
  TNR_TRY(reset_status(s));
  tnr_mpo A64;
  if (A->dtype == TNR_F32) {  // widened to float64 on the device, exactly
    TNR_TRY(widen_cores(s, *A, sb.widened, &A64));
    A = &A64;
  }

  // A' : merged operator
  tnr_mpo Am;
  memset(&Am, 0, sizeof(Am));
  Am.d = P.d;
  for (int i = 0; i < P.d; ++i) {
    Am.I[i] = P.I[i];
    Am.J[i] = P.J[i];
    Am.R[i] = P.RA[i];
    Am.core[i] = i == 0 ? nullptr : A->core[P.m - 1 + i];
  }
  Am.R[P.d] = 1;
  TNR_TRY(merge_leading(s, A, P, sb, &Am.core[0]));

  // Omega, Lemma 5.1
  {
    LaunchScope ls(K_OMEGA, s);
    k_omega<<<grid_for(P.omega_len), 256, 0, s>>>(seed, P.omega_len, sb.omega);
  }
  TNR_CK(cudaGetLastError());
  tnr_mpo Om;
  memset(&Om, 0, sizeof(Om));
  Om.d = P.d;
  {
    int64_t pos = 0;
    for (int i = 0; i < P.d; ++i) {
      Om.I[i] = P.J[i];
      Om.J[i] = i == 0 ? K : 1;
      Om.R[i] = 1;
      Om.core[i] = sb.omega + pos;
      pos += i == 0 ? P.J[0] * K : P.J[i];
    }
    Om.R[P.d] = 1;
  }
  tnr_mpo Y0, Y1;
  memset(&Y0, 0, sizeof(Y0));
  memset(&Y1, 0, sizeof(Y1));
  for (int i = 0; i < P.d; ++i) {
    Y0.core[i] = sb.P0[i];
    Y0.cap[i] = P.pcap[i];
    Y1.core[i] = sb.P1[i];
    Y1.cap[i] = P.pcap[i];
  }
  // Alg. 5.4
  // Mixed precision: the power-iteration products carry BF16 x3 noise (~1e-5 relative), so
  // their roundings truncate at tol_p = max(tol, kMixedTol); this perturbs range(Q) at 1e-4,
  // which moves the singular values of the FP64 Rayleigh-Ritz step B = Q^T A only at second
  // order (1e-8). B itself is rounded with the caller's tol in FP64.
  const bool mixed = o->precision == TNR_MIXED;
  const double tol_p = mixed ? std::max(o->tol, kMixedTol) : o->tol;
  TNR_TRY(contract_impl(s, Am, 0, Om, Y0, mixed));
  TNR_TRY(orthogonalize_impl(s, Y0, nullptr, tol_p, o->max_rank, sb.b, mixed));
  for (int it = 0; it < q; ++it) {
    TNR_TRY(contract_impl(s, Am, 1, Y0, Y1, mixed));
    TNR_TRY(orthogonalize_impl(s, Y1, nullptr, tol_p, o->max_rank, sb.b, mixed));
    TNR_TRY(contract_impl(s, Am, 0, Y1, Y0, mixed));
    TNR_TRY(orthogonalize_impl(s, Y0, nullptr, tol_p, o->max_rank, sb.b, mixed));
  }
  // B = Q^T A as Z = A^T Q, then Alg. 5.3
  TNR_TRY(contract_impl(s, Am, 1, Y0, Y1));
  {
    // V^(1) goes straight into the caller's V core 1.
    TNR_TRY(mpo_svd_impl(s, Y1, o->tol, o->max_rank, sb.b, sb.W, sb.S, V->core[0], k, V->cap[0]));
  }
  // Outputs. U = Q x_3 W^T on site 1 (Section 5.4), first k columns.
  {
    const int64_t I1 = Y0.I[0], t = Y0.R[1];
    if (I1 * k * t > U->cap[0]) return TNR_ENOMEM;
    TNR_TRY(gemm_f64(s, false, false, I1, k, K, 1.0, Y0.core[0], I1, I1 * K, sb.W, K, 0, 0.0, U->core[0], I1, I1 * k,
                     t));
  }
  U->R[0] = 1;
  V->R[0] = 1;
  U->R[1] = Y0.R[1];
  V->R[1] = Y1.R[1];
  U->I[0] = Y0.I[0];
  U->J[0] = k;
  V->I[0] = Y1.I[0];
  V->J[0] = k;
  for (int i = 1; i < P.d; ++i) {
    const int64_t ue = Y0.R[i] * Y0.I[i] * Y0.R[i + 1];
    const int64_t ve = Y1.R[i] * Y1.I[i] * Y1.R[i + 1];
    if (ue > U->cap[i] || ve > V->cap[i]) return TNR_ENOMEM;
    TNR_CK(cudaMemcpyAsync(U->core[i], Y0.core[i], sizeof(double) * ue, cudaMemcpyDeviceToDevice, s));
    TNR_CK(cudaMemcpyAsync(V->core[i], Y1.core[i], sizeof(double) * ve, cudaMemcpyDeviceToDevice, s));
    U->R[i + 1] = Y0.R[i + 1];
    V->R[i + 1] = Y1.R[i + 1];
    U->I[i] = Y0.I[i];
    V->I[i] = Y1.I[i];
    U->J[i] = 1;
    V->J[i] = 1;
  }
  TNR_CK(cudaMemcpyAsync(S, sb.S, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  return read_status(s);
}

}  // namespace

// Lemma 5.1 draws (the stream k_omega implements), for the differentiable solver.
int omega_fill(cudaStream_t s, uint64_t seed, int64_t count, double *out) {
  if (count <= 0) return TNR_OK;
  LaunchScope ls(K_OMEGA, s);
  k_omega<<<grid_for(count), 256, 0, s>>>(seed, count, out);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}
}  // namespace tnr

using namespace tnr;

extern "C" int tnr_mpo_contract(const tnr_mpo *A, int32_t trans, const tnr_mpo *X, tnr_mpo *Y, int32_t precision,
                                void *stream) {
  TNR_TRY(validate_input(A));
  TNR_TRY(validate_input(X));
  if (!Y || X->d != A->d || (trans != 0 && trans != 1)) return TNR_EINVAL;
  if (precision != TNR_FP64 && precision != TNR_MIXED) return TNR_EINVAL;
  for (int k = 0; k < A->d; ++k)
    if (!Y->core[k]) return TNR_EINVAL;
  return contract_impl((cudaStream_t)stream, *A, trans, *X, *Y, precision == TNR_MIXED);
}

namespace {
int orth_limits(const tnr_mpo *Y, Limits &L) {
  TNR_TRY(validate_input(Y));
  L = Limits();
  for (int k = 0; k < Y->d; ++k) {
    const int64_t rows = Y->R[k] * Y->I[k] * Y->J[k];
    L.maxcore = std::max(L.maxcore, core_elems(*Y, k));
    L.maxbond = std::max(L.maxbond, std::max(Y->R[k], Y->R[k + 1]));
    L.maxrows = std::max(L.maxrows, rows);
    if (k > 0) L.maxsq = std::max(L.maxsq, std::min(Y->R[k], Y->I[k] * Y->J[k] * Y->R[k + 1]));
  }
  L.maxsq = std::max(L.maxsq, Y->J[0]);
  L.maxcore = std::max(L.maxcore, Y->I[0] * Y->J[0] * L.maxbond);
  if (L.maxsq > 1024) return TNR_ENOMEM;
  return TNR_OK;
}
}  // namespace

extern "C" int tnr_orthogonalize_workspace(const tnr_mpo *Y, size_t *bytes) {
  Limits L;
  TNR_TRY(orth_limits(Y, L));
  if (!bytes) return TNR_EINVAL;
  Arena ar;
  Bufs b;
  carve(ar, L, b);
  *bytes = ar.off;
  return TNR_OK;
}

extern "C" int tnr_orthogonalize(tnr_mpo *Y, double *R_KxK, const tnr_opts *opts, void *ws, size_t ws_bytes,
                                 void *stream) {
  Limits L;
  if (opts && opts->rounding != TNR_ROUND_TWO_SWEEP) return TNR_EINVAL;
  TNR_TRY(orth_limits(Y, L));
  for (int k = 1; k < Y->d; ++k)
    if (Y->J[k] != 1) return TNR_EINVAL;
  if (Y->I[0] < Y->J[0]) return TNR_EINVAL;  // Alg. 5.2 needs I_1 >= K
  Arena ar;
  ar.base = static_cast<char *>(ws);
  ar.size = ws_bytes;
  Bufs b;
  carve(ar, L, b);
  if (!ar.ok || !ws) return TNR_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  TNR_TRY(reset_status(s));
  const double tol = opts ? opts->tol : 0.0;
  const int64_t mr = opts ? opts->max_rank : 0;
  TNR_TRY(orthogonalize_impl(s, *Y, R_KxK, tol, mr, b));
  return read_status(s);
}

extern "C" int tnr_solve_query(const tnr_mpo *A, int32_t k, int32_t p, const tnr_opts *opts, tnr_mpo *U_shape,
                               tnr_mpo *V_shape, size_t *ws_bytes) {
  if (k < 1 || p < 0 || !opts) return TNR_EINVAL;
  const int64_t K = (int64_t)k + p;
  Plan P;
  TNR_TRY(make_plan(A, K, opts, P));
  if (opts->rounding == TNR_ROUND_TWO_SWEEP) {
    Arena ar;
    SolveBufs sb;
    carve_solve(ar, P, K, sb, A);
    if (ws_bytes) *ws_bytes = ar.off;
  } else if (ws_bytes) {
    *ws_bytes = 0;  // zip-up runs in the persistent batch, whose workspace tnr_batch_workspace gives
  }
  for (tnr_mpo *M : {U_shape, V_shape}) {
    if (!M) continue;
    const bool isU = M == U_shape;
    M->d = P.d;
    for (int i = 0; i < P.d; ++i) {
      M->I[i] = isU ? P.I[i] : P.J[i];
      M->J[i] = i == 0 ? k : 1;
      M->R[i] = P.sq[i];
      M->cap[i] = P.sq[i] * M->I[i] * (i == 0 ? k : 1) * P.sq[i + 1];
      M->core[i] = nullptr;
    }
    M->R[P.d] = 1;
  }
  return TNR_OK;
}

extern "C" int tnr_solve(const tnr_mpo *A, int32_t k, int32_t p, int32_t q, uint64_t seed, const tnr_opts *opts,
                         tnr_mpo *U, double *S, tnr_mpo *V, void *ws, size_t ws_bytes, void *stream) {
  return solve_impl((cudaStream_t)stream, A, k, p, q, seed, opts, U, S, V, ws, ws_bytes);
}
