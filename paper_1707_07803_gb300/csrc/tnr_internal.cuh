// Internal helpers shared by the translation units of libtnrsvd.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/tnrsvd.h"

namespace tnr {

// Device status words (per device and host-thread slot, in runtime.cu): the first device-side
// failure in a slot wins.
// Kernels receive its address; status_ptr() returns it for the current device and the calling
// host thread's slot (set_status_slot; 0 unless the thread is a batched-solve worker).
constexpr int kStatusSlots = 64;
// Per-device caches of device-symbol addresses (status words, compiled-in scratch) cover the
// first kMaxDevices device ordinals; a call on a higher ordinal fails with TNR_ERANGE/ECUDA.
constexpr int kMaxDevices = 64;
int *status_ptr();
void set_status_slot(int slot);

__device__ __forceinline__ void set_status(int *st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Iteration cap for every spin-wait on a flag written by another CTA. At ~1e3 cycles per
// poll this bounds a wait to roughly a second at 2 GHz.
constexpr long long kSpinCap = 2000000;

// Kernel classes for launch counting and event timing.
enum KClass : int {
  K_CONV_ROWPTR = 0,
  K_CONV_FLAGS,
  K_CONV_SCAN,
  K_CONV_FILL,
  K_OMEGA,
  K_MERGE,
  K_CONTRACT,
  K_CONTRACT_TC,
  K_GEMM,
  K_QR,        // multi-CTA Householder QR (k_qr_coop, k_qrcp)
  K_QR_SMALL,  // one-CTA unpivoted QR (k_qr_small, k_qr_small_tpc)
  K_QR_PIV,    // one-CTA column-pivoted QR of the compression sweep
  K_SVD,
  K_MISC,
  K_ROUND,     // fused one-CTA rounding sweeps (k_round_small)
  K_DIFF,      // differentiable solver: tape forward and adjoint kernels
  K_BATCH,     // persistent batched solver (one CTA per problem)
  K_NUM_CLASSES
};

// Launch bookkeeping: call before/after each kernel launch on `s`.
void stats_begin(int cls, cudaStream_t s);
// Add algorithmic work (flops or bytes, per class) for the launch being recorded.
void stats_work(int cls, double work);
void stats_end(int cls, cudaStream_t s);

struct LaunchScope {
  int cls;
  cudaStream_t s;
  LaunchScope(int c, cudaStream_t st) : cls(c), s(st) { stats_begin(cls, s); }
  ~LaunchScope() { stats_end(cls, s); }
};

// Bump allocator over the caller's workspace; with base == nullptr it only measures.
struct Arena {
  char *base = nullptr;
  size_t size = 0;
  size_t off = 0;
  bool ok = true;
  template <typename T>
  T *take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    size_t at = off;
    off += bytes;
    if (base == nullptr) return nullptr;
    if (off > size) {
      ok = false;
      return nullptr;
    }
    return reinterpret_cast<T *>(base + at);
  }
};

int check_cuda(cudaError_t e);
int check_cuda_at(cudaError_t e, const char *file, int line);  // same, naming the call site
// Raises (never lowers) a kernel's dynamic shared-memory limit on the current device.
int ensure_dynamic_smem(const void *func, size_t bytes);
int read_status(cudaStream_t s);  // synchronises s, returns and clears the device status word
// Copies device regions to host memory and reads (and clears) the status word with one
// synchronisation of s (pinned staging); returns the status.
struct ReadBack {
  void *dst;
  const void *src;
  size_t bytes;
};
int read_back(cudaStream_t s, const ReadBack *items, int n);
// The same read-back without any staging buffer: plain copies into the caller's (pageable) host
// memory and one synchronisation of s. Allocates nothing, on the host or on the device.
int read_back_unstaged(cudaStream_t s, const ReadBack *items, int n);
int reset_status(cudaStream_t s);

#define TNR_CK(expr)                                           \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return tnr::check_cuda_at(_e, __FILE__, __LINE__); \
  } while (0)

#define TNR_TRY(expr)           \
  do {                          \
    int _rc = (expr);           \
    if (_rc != TNR_OK) return _rc; \
  } while (0)

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Compression cutoff relative to ||M_k||_F: the rounding level of the product that made Y.
// FP64 products: min(64 eps, tol / 100). BF16 x3 products carry about 2^-16 relative error per
// term, so their noise directions are dropped at 0.05 tol (tol is then at least kMixedTol).
constexpr double kMixedTol = 1.2e-4;
// The persistent batch's products use FP32 operands (about 2^-24 relative per term, ~1e-7 noise in
// a product): its power iteration is rounded at max(tol, kMixedTolF32), an order above that noise.
constexpr double kMixedTolF32 = 1e-6;
__host__ __device__ inline double compress_cut(double tol, bool mixed_product) {
  if (mixed_product) return 0.05 * tol;
  const double a = 64.0 * 2.220446049250313e-16, b = 0.01 * tol;
  return a < b ? a : b;
}

// ---- Solve plan (host) ----

// Buffer-size bounds of one orthogonalisation / solve.
struct Limits {
  int64_t maxcore = 1;  // elements of the largest core
  int64_t maxbond = 1;  // largest bond
  int64_t maxrows = 1;  // largest row count of an L->R QR
  int64_t maxsq = 1;    // largest square factor side
};

// The merged operator A' (Section 6.3) and the plan of every buffer of a solve.
struct Plan {
  int m = 1;  // sites merged into site 1
  int d = 0;  // sites after the merge
  int64_t I[TNR_MAX_SITES], J[TNR_MAX_SITES], RA[TNR_MAX_SITES + 1];
  int64_t sq[TNR_MAX_SITES + 1];  // cap of Q bonds (max of the I- and J-side bounds)
  int64_t pcap[TNR_MAX_SITES];    // product core capacity
  int64_t omega_len = 0;
  int64_t merged_elems = 0;
  Limits L;
};

// Dims, ranks and core pointers of an input MPO; allow_f32: TNR_F32 cores are accepted.
int validate_input(const tnr_mpo *A, bool allow_f32 = false);
// Element count of every core of A (for the float64 copies of TNR_F32 inputs).
int64_t mpo_elems(const tnr_mpo &A);
// Widens A's float32 cores into float64 buffers (dst[k] holds core k); *out = A with those cores.
int widen_cores(cudaStream_t s, const tnr_mpo &A, double *const *dst, tnr_mpo *out);
// y (float32) <- x (float64), n elements (round to nearest).
int narrow_to_f32(cudaStream_t s, const double *x, float *y, int64_t n);
// Merge count, merged dimensions, bond caps (Thm 3.2 bounds and max_rank) and buffer bounds of
// a solve with K = k + p columns.
int make_plan(const tnr_mpo *A, int64_t K, const tnr_opts *o, Plan &P);

// ---- FP64 dense building blocks (column-major, explicit leading dimensions) ----

// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], b = 0..batch-1 with element strides sa, sb, sc.
int gemm_f64(cudaStream_t s, bool transA, bool transB, int64_t m, int64_t n, int64_t k, double alpha,
             const double *A, int64_t lda, int64_t sa, const double *B, int64_t ldb, int64_t sb, double beta,
             double *C, int64_t ldc, int64_t sc, int64_t batch = 1);

// Thin Householder QR of the m x n matrix A (lda): A <- Q (m x min(m,n), explicit), Rout <- R
// (min(m,n) x n, upper trapezoidal, ldr). Scratch from the arena: V (m x n), tau, flags.
size_t qr_f64_scratch(int64_t m, int64_t n);
// Scratch enough for any QR of an m x n matrix with m * n <= max_elems and n <= max_n.
size_t qr_scratch_bound(int64_t max_elems, int64_t max_n);
int qr_f64(cudaStream_t s, double *A, int64_t m, int64_t n, int64_t lda, double *Rout, int64_t ldr,
           void *scratch);

// Rank-revealing QR with noise cutoff (column pivoting): A <- Q (m x r, explicit), Rout <- R
// = Q^T A (r x n, original column order, ldr >= min(m, n)); r written to *r_dev (device).
// Directions whose residual column norm is <= cut_rel * ||A||_F are dropped (r >= 1).
// *used = false when the matrix does not fit the shared-memory layout (nothing launched).
size_t qrcp_scratch(int64_t m, int64_t n);
size_t qrcp_scratch_bound(int64_t max_elems, int64_t max_n);
int qrcp_f64(cudaStream_t s, double *A, int64_t m, int64_t n, int64_t lda, double *Rout, int64_t ldr, double cut_rel,
             void *scratch, int64_t *r_dev, bool *used);

// Small-matrix Householder QR in one CTA (matrix in shared memory): A = op(src) (m x n);
// optional column pivoting with a cutoff (see k_qr_small). Q (m x r) written as Q or Q^T,
// R = Q^T A (r x n, original column order) written as R or R^T; r to *r_dev (may be null when
// not pivoting: r = min(m, n)). The source is read completely before any output is written,
// so Q or R may overwrite it. ldq <= 0 packs Q^T with leading dimension r (known on device).
bool qr_small_fits(int64_t m, int64_t n);
int qr_small_f64(cudaStream_t s, const double *src, int64_t lds, int64_t m, int64_t n, bool trans_src, bool pivot,
                 double cut_rel, double *Q, int64_t ldq, bool trans_q, double *R, int64_t ldr, bool trans_r,
                 int64_t *r_dev);

// SVD of the n x n matrix G (ldg) by one-sided Jacobi: G <- U (columns), S (descending),
// V (n x n, ldv) with G_in = U diag(S) V^T. `sweeps_out` (device int, may be null).
size_t jacobi_scratch(int64_t n);
int jacobi_svd_f64(cudaStream_t s, double *G, int64_t n, int64_t ldg, double *S, double *V, int64_t ldv,
                   void *scratch);

// Tensor-core (tcgen05, BF16 in / FP32 accumulate) site-1 product; see contract_tc.cu.
int contract_site1_tc(cudaStream_t s, const double *A, int64_t I, int64_t J, int64_t R2, const double *X, int64_t Kx,
                      int64_t S2, int trans, double *Y, bool split);

// Fused truncated-SVD step of the right-to-left sweep for a core M (t x w) that fits one CTA:
// writes V^T[:r] (r x w, ld r; may alias M) and U[:, :r] diag(S) (t x r, ld t) and r (device).
size_t svd_step_smem(int64_t t, int64_t w);
int svd_step_small(cudaStream_t s, const double *M, int64_t t, int64_t w, const double *norm2, double tol,
                   int64_t dm1, int64_t max_rank, double *core_out, double *US, int64_t *r_dev);

// Both rounding sweeps (L->R QR, R->L truncated SVD) of Y in one one-CTA launch when every core
// fits shared memory; see round_small.cu. Leaves *launched false (nothing queued) otherwise.
constexpr size_t kRoundSmallMaxSmem = 200 * 1024;
// certify: cores 1..d-1 are right-orthonormal on entry (after the exact compression), which lets
// the kernel skip both sweeps when it can show that no bond would be truncated.
int round_small(cudaStream_t s, const tnr_mpo &Y, double tol, int64_t max_rank, bool certify, int64_t *R_dev,
                bool *launched);

// CholeskyQR2 of the site-1 matrix (I1 t) x K of core0 (1, I1, K, t) in one cooperative launch
// (site1_qr.cu): Q~ to Qout (column-major) or back into core0 (core_out), R~ to Rout; *flag
// (device) = 1 when the factorisation must be redone by Householder. t_dev (may be null): the
// rank in device memory, t then being its upper bound; gate (may be null): run only when *gate
// != 0 on the device. *launched = false when the sizes are outside its layout.
int site1_cholqr2(cudaStream_t s, double *core0, int64_t I1, int64_t K, int64_t t, const int64_t *t_dev, bool core_out,
                  const int *gate, double *Q1, int64_t q1cap, double *G, double *Rout, double *Qout, int *flag,
                  unsigned *bar, bool *launched);

// Lemma 5.1 normal draws (SplitMix64 + Box-Muller), `count` values in draw order.
int omega_fill(cudaStream_t s, uint64_t seed, int64_t count, double *out);

// Exact right-to-left compression of a product MPO as one cooperative kernel (compress_coop.cu),
// queued without a read-back; with fuse_round a complete compression is followed by the fused
// rounding sweeps in the same launch (ctl[2] = 1 when they ran). ctl[0]: the first bond left to the
// host-driven sweep (0: none); R_dev: the ranks of the bonds the device finished.
int compress_launch(cudaStream_t s, const tnr_mpo &Y, double cut, double *L, double *buf0, double *buf1,
                    int64_t cap_buf, unsigned *bar, int *ctl, int64_t *R_dev, bool fuse_round, double tol,
                    int64_t max_rank, int64_t *R_round, bool *launched);
// CTAs per factoring cluster of the compression (1: one-CTA QR, or before the first launch).
int compress_cluster_size();
// Records the algorithmic work of the bonds the device compressed, from the ranks h read back.
void compress_record_work(const tnr_mpo &Y, const int64_t *h, int first_host_bond);

// Small element-wise kernels.
int copy_matrix_f64(cudaStream_t s, const double *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t n,
                    bool transpose);
int scale_columns_f64(cudaStream_t s, double *A, int64_t lda, int64_t m, int64_t n, const double *scale);

}  // namespace tnr
