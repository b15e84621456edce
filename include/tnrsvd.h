/*
 * tnrsvd.h - C ABI of the GB300 TNrSVD library (libtnrsvd.so).
 *
 * Implements the data-parallel path of "Computing low-rank approximations of large-scale
 * matrices with the Tensor Network randomized SVD" (Batselier, Yu, Daniel, Wong):
 * sparse matrix -> MPO conversion (Alg. 4.1), the MPO x MPO product (Section 5.2), MPO-QR
 * with integrated rounding (Alg. 5.2 and Section 5.4), MPO-SVD (Alg. 5.3) and the randomized
 * MPO subspace iteration (Alg. 5.4) that drives the rSVD of Alg. 5.1.
 *
 * Conventions (Section 2, Eq. (2.1); Section 3):
 *  - Row and column multi-indices are column-major: row = i_1 + I_1 (i_2 + I_2 (i_3 + ...)).
 *  - Core k of an MPO is R_k x I_k x J_k x R_{k+1}, stored contiguously in column-major order:
 *    element (r, i, j, r') at offset r + R_k (i + I_k (j + J_k r')). R_1 = R_{d+1} = 1.
 *  - A tall I x K matrix (Y, Q, U, V of Section 5) is an MPO whose site-1 core is
 *    1 x I_1 x K x R_2 and whose other cores have J_k = 1 (Lemma 5.1, Algs. 5.2-5.3).
 *  - All floating-point data is IEEE float64 unless a precision mode says otherwise.
 *
 * Ownership: the caller allocates every device buffer (cores, outputs, workspace) and owns
 * it; the library never allocates device memory. Host-side descriptors are read during the
 * call only. Work is enqueued on the caller's stream; calls that return host values
 * (ranks, counts) synchronise that stream.
 *
 * Errors: every entry point returns TNR_OK (0) or a negative status. Argument errors are
 * detected before any work is enqueued. Device-side failures (non-finite data, an exhausted
 * bounded wait, an unsorted or duplicate COO entry) are recorded in a device status word and
 * reported by the next call that synchronises. tnr_strerror() names a status.
 */
#ifndef TNRSVD_H
#define TNRSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TNR_MAX_SITES 64

enum tnr_status {
  TNR_OK = 0,
  TNR_EINVAL = -1,      /* inconsistent dims/ranks, K too large, bad pointer or size */
  TNR_EDUP = -2,        /* duplicate (row, col) entry in the COO input */
  TNR_ENOTSORTED = -3,  /* COO input not sorted by (row, col) */
  TNR_ENONFINITE = -4,  /* NaN or Inf met in device data */
  TNR_ENOMEM = -5,      /* workspace or output capacity too small */
  TNR_ECUDA = -6,       /* a CUDA runtime call failed */
  TNR_ETIMEOUT = -7,    /* a bounded device wait ran out */
  TNR_ERANGE = -8       /* an index or count exceeds the supported range */
};

enum tnr_precision {
  TNR_FP64 = 0,  /* every step in float64 */
  TNR_MIXED = 1  /* products A*Omega, A^T Q, A Q with reduced-precision operands and FP32
                    accumulation, B = Q^T A, its rounding with tol, the QR sweeps and the SVDs in
                    float64. Single solve (tnr_solve, tnr_solve_batched): BF16 x3 operands (about
                    2^-16 relative; the dense site-1 products on tcgen05 tensor cores), the
                    power iteration rounded at max(tol, 1.2e-4). Persistent batch (tnr_batch_*):
                    FP32 operands on the FP32 pipe (about 2^-24 relative, one FMA per term), the
                    power iteration rounded at max(tol, 1e-6). The tolerances sit above each
                    product's noise level, so the rounding does not keep noise directions. */
};

/* Element type of an MPO's cores. Outputs are always TNR_F64. TNR_F32 inputs are accepted by
 * tnr_solve / tnr_solve_query (A) and tnr_diff_forward / tnr_diff_backward (A, dA): the cores
 * are widened to float64 on the device (exactly) before the method runs; every other entry point
 * requires TNR_F64 (TNR_EINVAL otherwise). */
enum tnr_dtype { TNR_F64 = 0, TNR_F32 = 1 };

/* MPO descriptor (host memory). For inputs only d, dtype, I, J, R and core are read. For
 * outputs the caller sets d, I, J, core and cap (capacity of each core buffer in elements); the
 * library writes the achieved ranks into R. */
typedef struct tnr_mpo {
  int32_t d;
  int32_t dtype; /* enum tnr_dtype; 0 (TNR_F64) for every buffer the library writes */
  int64_t I[TNR_MAX_SITES];
  int64_t J[TNR_MAX_SITES];
  int64_t R[TNR_MAX_SITES + 1];
  double *core[TNR_MAX_SITES];
  int64_t cap[TNR_MAX_SITES];
} tnr_mpo;

/* How a product is rounded (Section 5.4 integrates SVD-based rounding with the MPO-QR sweep).
 * TNR_ROUND_TWO_SWEEP: the product op(A) X is formed in full (ranks R_k S_k), then orthogonalised:
 *   left-to-right QR sweep, right-to-left truncating SVD sweep, site-1 step of Alg. 5.2/5.3.
 * TNR_ROUND_ZIPUP (truncate as you go): the product is rounded while it is formed, right to left:
 *   at site k the product core, with the factor carried from site k+1 absorbed into its right bond,
 *   is the (R_k S_k) x (n_k K_k t_{k+1}) matrix T_k; its SVD keeps the smallest r >= 1 with
 *   sum_{l>r} s_l^2 <= tol^2 ||T_k||_F^2 / (d-1) (then r <= max_rank), core k becomes the r kept
 *   right singular vectors and U diag(s) is carried to site k-1; site 1 absorbs the last factor.
 *   The product cores are never formed. The result is then orthogonalised as above (on bonds of
 *   at most max_rank). Accepted by the persistent batched solver (tnr_batch_*); the other entry
 *   points require TNR_ROUND_TWO_SWEEP (TNR_EINVAL otherwise). */
enum tnr_rounding { TNR_ROUND_TWO_SWEEP = 0, TNR_ROUND_ZIPUP = 1 };

/* Rounding options (Section 5.4 integrates SVD-based rounding with the MPO-QR sweep).
 * At each bond the smallest rank r >= 1 is kept whose discarded singular values satisfy
 * sum s_l^2 <= delta^2, delta = tol * ||Y||_F / sqrt(d - 1); then r <= max_rank if max_rank > 0. */
typedef struct tnr_opts {
  int32_t precision;  /* enum tnr_precision */
  int32_t rounding;   /* enum tnr_rounding */
  double tol;
  int64_t max_rank;   /* 0: only the structural bounds of Thm 3.2 apply */
} tnr_opts;

/* ---------------------------------------------------------------------------------------
 * Sparse -> MPO conversion, Alg. 4.1 (Section 4). The result is the block form of the
 * rank-R MPO of Lemma 4.2: R nonzero I_1 x J_1 blocks X_t (column-major, block t at
 * X + t*I_1*J_1, which is core A^(1)(0, i_1, j_1, t)), and for each block the digits
 * i_2, j_2, ..., i_d, j_d of its block-row p and block-column q (mixed radix, site 2
 * fastest) as uint8, row t of a R x 2(d-1) array. Blocks are ordered by (p, q), p major.
 *
 * Inputs: row, col (int64, device), val (float64, device), nnz entries sorted by (row, col)
 * with no duplicates; nrows = prod I, ncols = prod J; I_1 * J_1 <= 4096, I_k, J_k <= 256
 * for k >= 2; nnz < 2^31. Two phases (Section 4.2: the sizes are known a priori, so the
 * caller preallocates): tnr_sparse_count() writes R to *R_out (synchronises); the caller
 * allocates X (R*I_1*J_1 doubles) and digits (R*2(d-1) bytes); tnr_sparse_fill() writes
 * them. Both take the same workspace, of at least tnr_sparse_workspace() bytes, whose
 * contents must survive from count to fill. Errors: TNR_EINVAL (dims), TNR_ENOTSORTED,
 * TNR_EDUP, TNR_ERANGE (an index outside the matrix), TNR_ENOMEM (workspace too small).
 * ------------------------------------------------------------------------------------- */
int tnr_sparse_workspace(int64_t nrows, int64_t ncols, int64_t nnz, int32_t d, const int64_t *I,
                         const int64_t *J, size_t *bytes);
int tnr_sparse_count(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row, const int64_t *col,
                     int32_t d, const int64_t *I, const int64_t *J, int64_t *R_out, void *ws,
                     size_t ws_bytes, void *stream);
int tnr_sparse_fill(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row, const int64_t *col,
                    const double *val, int32_t d, const int64_t *I, const int64_t *J, int64_t R,
                    double *X, uint8_t *digits, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------------------
 * Dense cores of the Alg. 4.1 MPO from its block form (Section 4.1, Eq. (4.1): the sum of the
 * rank-1 MPOs E^(d)_{i_d j_d} (x) ... (x) E^(2)_{i_2 j_2} (x) X_t, rank R at every bond by
 * Lemma 4.2), for rounding the converted MPO (Section 4.2's example: a Kronecker product of
 * three 2 x 2 matrices converts to rank 16 and rounds to rank 1; Section 6.1 rounds a converted
 * MPO from rank 347 to 7). Core 1 (1 x I_1 x J_1 x R) holds the blocks (core(0, i1, j1, t) =
 * X_t(i1, j1)); core k = 2..d-1 (R x I_k x J_k x R) is the bond-diagonal selection
 * core(t, i, j, t) = [i = i_{t,k}][j = j_{t,k}]; core d (R x I_d x J_d x 1) likewise with the bond
 * closed; with d = 1 the single core is the sum of the blocks. Inputs R, X, digits as written by
 * tnr_sparse_fill (device). Output: A->core[k] (device) with room A->cap[k] elements each, set by
 * the caller; the library sets A->d, dtype, I, J, R. Copy and integer work only (bit-exact).
 * Asynchronous on `stream`; a digit outside its site's range is reported through the device
 * status word (TNR_ERANGE at the next synchronising call). Errors: TNR_EINVAL (dims, pointers,
 * R < 1), TNR_ENOMEM (a core capacity too small), TNR_ERANGE (I_1 J_1 > 4096 or R >= 2^31).
 * Interior cores take R^2 I_k J_k doubles: this serves converted MPOs of modest rank.
 * ------------------------------------------------------------------------------------- */
int tnr_sparse_cores(int64_t R, const double *X, const uint8_t *digits, int32_t d, const int64_t *I,
                     const int64_t *J, tnr_mpo *A, void *stream);

/* ---------------------------------------------------------------------------------------
 * Sparse -> MPO conversion that allocates nothing. The paper has no counterpart: this entry is
 * a service to callers of this library. It computes exactly what tnr_sparse_count followed by
 * tnr_sparse_fill computes, for callers that cannot call cudaMalloc or take memory from an
 * allocator: for example a plug-in loaded into a host process whose own memory manager has
 * reserved all of the device memory up front (a second allocator would fail or fragment it),
 * or code that must not pay the device-wide synchronisation an allocation can cause. Instead
 * of a caller workspace it uses a scratch array compiled into the library, sized for at most
 * TNR_NOALLOC_MAX_NNZ nonzeros (32 MiB + 32 KiB, held on every GPU that loads the library
 * until the process exits). Neither device memory nor host memory is allocated by the call
 * (R is copied straight into the caller's int64, without a pinned staging buffer).
 *
 * Inputs as for tnr_sparse_count/fill. The caller passes the outputs: X with room for
 * max_blocks*I_1*J_1 doubles and digits with room for max_blocks*2(d-1) bytes; each nonzero
 * opens at most one block, so max_blocks = nnz always suffices. *R_out receives the number of
 * blocks R. Errors: TNR_ERANGE when nnz > TNR_NOALLOC_MAX_NNZ (nothing enqueued);
 * TNR_ENOMEM when R > max_blocks (X and digits untouched); otherwise as tnr_sparse_count.
 * The call synchronises the stream once, to read R; the fill is then enqueued asynchronously.
 * The first call on a device looks the scratch address up (cudaGetSymbolAddress with that
 * device current). Every call shares the scratch, which keeps the previous call's contents
 * (each call writes every entry it reads); calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller. With the library's
 * instrumentation switched on (tnr_stats_enable; off by default) the call records timing
 * events like every other entry point.
 * ------------------------------------------------------------------------------------- */
#define TNR_NOALLOC_MAX_NNZ 8388608
int tnr_sparse_to_mpo_noalloc(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row, const int64_t *col,
                              const double *val, int32_t d, const int64_t *I, const int64_t *J, double *X,
                              uint8_t *digits, int64_t max_blocks, int64_t *R_out, void *stream);

/* ---------------------------------------------------------------------------------------
 * MPO x MPO product, Section 5.2: Y = op(A) X with op(A) = A (trans = 0) or A^T (trans = 1).
 * X is a tall matrix MPO (site 1: 1 x n_1 x K x S_2, others S_k x n_k x 1 x S_{k+1}) whose
 * row dims n_k equal J_k (trans = 0) or I_k (trans = 1). Per site
 *   Y_k((r,s), i, c, (r',s')) = sum_j A_k(r,i,j,r') X_k(s,j,c,s')     (trans = 0)
 * with product bonds numbered r + R_k s; ranks multiply. Y's descriptor: the caller sets
 * core and cap; the library sets d, I, J, R. precision = TNR_FP64: FP64 arithmetic.
 * precision = TNR_MIXED: every operand is rounded to BF16 as hi + lo (hi = bf16(x),
 * lo = bf16(x - hi)) and the products hi*hi + hi*lo + lo*hi are accumulated in FP32 (about
 * 1e-5 relative per product); dense sites (both outer bonds 1, shared dim >= 16) run on the
 * tcgen05 tensor cores. Errors: TNR_EINVAL, TNR_ENOMEM.
 * ------------------------------------------------------------------------------------- */
int tnr_mpo_contract(const tnr_mpo *A, int32_t trans, const tnr_mpo *X, tnr_mpo *Y, int32_t precision, void *stream);

/* ---------------------------------------------------------------------------------------
 * MPO-QR with integrated rounding, Alg. 5.2 + Section 5.4, in place: Y (a tall matrix MPO,
 * K columns on site 1, I_1 >= K) becomes Q with Q^T Q = I_K, and R_KxK (device, K*K
 * doubles, column-major, upper triangular) receives R with Y = Q R up to the rounding.
 * Steps: left-to-right Householder QR sweep (R factors absorbed to the right), right-to-left
 * truncating SVD sweep (the rule of tnr_opts), then the site-1 QR of Alg. 5.2. Y's ranks
 * are updated in Y->R. ws: at least tnr_orthogonalize_workspace() bytes. Synchronises.
 * ------------------------------------------------------------------------------------- */
int tnr_orthogonalize_workspace(const tnr_mpo *Y, size_t *bytes);
int tnr_orthogonalize(tnr_mpo *Y, double *R_KxK, const tnr_opts *opts, void *ws, size_t ws_bytes,
                      void *stream);

/* ---------------------------------------------------------------------------------------
 * TNrSVD, Alg. 5.4 + Alg. 5.3 driving Alg. 5.1: rank-k approximation A ~= U diag(S) V^T of
 * the MPO A with oversampling p (K = k + p) and q power iterations. Leading sites are merged
 * until I_1 >= K and J_1 >= K (Section 6.3); the random MPO Omega of Lemma 5.1 is drawn on
 * the device from `seed` (SplitMix64 counter stream, Box-Muller normals; Omega^(1) first in
 * column-major order, then the site vectors). Outputs: U (rows I, k columns on site 1) and
 * V (rows J, k columns on site 1) over the merged sites, S (k doubles, device, descending).
 * tnr_solve_query() fills the merged d, I, J and the per-core capacities (upper bounds) of U
 * and V, and the workspace size; the caller allocates and sets U->core, V->core. On return
 * U->R and V->R hold the achieved ranks. Synchronises (ranks are read back per bond).
 * Errors: TNR_EINVAL (K > prod I or prod J, k < 1, q < 0), TNR_ENOMEM, TNR_ENONFINITE.
 * ------------------------------------------------------------------------------------- */
int tnr_solve_query(const tnr_mpo *A, int32_t k, int32_t p, const tnr_opts *opts, tnr_mpo *U_shape,
                    tnr_mpo *V_shape, size_t *ws_bytes);
int tnr_solve(const tnr_mpo *A, int32_t k, int32_t p, int32_t q, uint64_t seed, const tnr_opts *opts,
              tnr_mpo *U, double *S, tnr_mpo *V, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------------------
 * Batched TNrSVD: n independent problems (each exactly as tnr_solve: its own A, k, p, q,
 * seed, options and caller-allocated outputs U, S, V) solved concurrently on the current
 * device. The paper solves one matrix at a time; this entry serves many small MPOs, whose
 * solves are chains of short, mostly one-SM kernels that leave most of the GPU idle when run
 * one after another. `workers` host threads (0: min(n, 16); at most 63) each drive their own
 * CUDA stream and take problems from a shared counter; worker w uses the workspace slice
 * ws + w * ws_stride (ws_stride: at least the largest tnr_solve_query workspace of the
 * batch, a multiple of 256; ws holds workers * ws_stride bytes) and its own device status
 * word, so one problem's device-side error never reaches another. The batch starts after
 * the work already queued on `stream` and `stream` waits for the whole batch; the call
 * returns when every problem is done. Each problem's status is written to its `status`;
 * the return value is the first non-zero status in index order (TNR_OK when all succeed),
 * or TNR_EINVAL for bad batch arguments (nothing is solved then).
 * ------------------------------------------------------------------------------------- */
typedef struct {
  const tnr_mpo *A;
  int32_t k, p, q, reserved;
  uint64_t seed;
  tnr_opts opts;
  tnr_mpo *U;
  double *S;
  tnr_mpo *V;
  int32_t status; /* out */
  int32_t reserved2;
} tnr_problem;
int tnr_solve_batched(int32_t n, tnr_problem *probs, int32_t workers, void *ws, size_t ws_stride, void *stream);

/* ---------------------------------------------------------------------------------------
 * Persistent batched TNrSVD: the same n independent problems (tnr_problem above, the same
 * steps as tnr_solve: Alg. 5.4 with Algs. 5.2/5.3, merge of Section 6.3, Omega of Lemma 5.1,
 * rounding of Section 5.4) solved by ONE kernel launch in which each CTA runs the whole
 * pipeline of one problem and takes the next problem from a device work queue. Ranks stay on
 * the device; nothing goes back to the host until the batch is done, so the launch can be
 * captured in a CUDA graph and replayed.
 *   tnr_batch_workspace: bytes of device workspace for the batch (descriptors and every
 *     problem's scratch at its structural rank bounds).
 *   tnr_batch_create: validates and plans every problem (errors as tnr_solve; nothing is
 *     launched for an invalid batch), uploads the descriptors into ws (synchronises `stream`),
 *     and chooses the launch configuration. flags: bit 0 = autotune the CTAs per SM for this
 *     shape bucket by timing the batch (once per process and bucket; the batch is solved
 *     while tuning), bit 1 = capture the launch in a CUDA graph, bits 4-7 = CTAs per SM set by
 *     the caller (1..15; overrides bit 0; fewer are used if they do not fit). `probs`, the MPOs and output
 *     buffers they point to, and ws must stay valid until tnr_batch_destroy. *handle receives
 *     an opaque host handle.
 *   tnr_batch_launch: queues the batch on `stream` (a graph launch when captured). Reads A,
 *     writes every U, S, V; it may be repeated (each launch solves the batch again).
 *   tnr_batch_collect: synchronises `stream`, writes each problem's status and the shapes and
 *     ranks of its U and V (as tnr_solve does); returns the first non-zero status in queue
 *     order, TNR_OK when all succeeded.
 *   tnr_batch_config: the chosen grid, CTAs per SM and dynamic shared memory per CTA.
 *   tnr_batch_destroy: frees the handle (not ws).
 * Device-side errors are per problem (TNR_ENOMEM: an output capacity too small; TNR_ENONFINITE;
 * TNR_ERANGE: a work area beyond the planned bound).
 * ------------------------------------------------------------------------------------- */
int tnr_batch_workspace(int32_t n, const tnr_problem *probs, size_t *bytes);
int tnr_batch_create(int32_t n, tnr_problem *probs, int32_t flags, void *ws, size_t ws_bytes, void *stream,
                     void **handle);
int tnr_batch_launch(void *handle, void *stream);
int tnr_batch_collect(void *handle, void *stream);
int tnr_batch_config(void *handle, int32_t *grid, int32_t *ctas_per_sm, int64_t *smem_bytes);
int tnr_batch_destroy(void *handle);

/* ---------------------------------------------------------------------------------------
 * Self-test of the bounded device waits (no counterpart in the paper). Every spin-wait of the
 * library's kernels on work of another CTA (grid barriers, mbarriers) is capped and reports
 * TNR_ETIMEOUT instead of waiting forever. This entry makes such a wait run out on purpose: two
 * CTAs enter a grid barrier, one returns without arriving, the other gives up after spin_cap
 * polls (1 <= spin_cap <= the library's cap). Returns TNR_ETIMEOUT (the expected outcome; the
 * device status word is cleared again and the context stays usable), TNR_OK if the wait somehow
 * completed, TNR_EINVAL for a bad cap. Synchronises `stream`.
 * ------------------------------------------------------------------------------------- */
int tnr_selftest_wait_timeout(int64_t spin_cap, void *stream);

/* ---------------------------------------------------------------------------------------
 * TNrSVD of a sparse matrix given in the block form of Alg. 4.1 (R, X, digits as produced by
 * tnr_sparse_fill; any block order). The MPO of Alg. 4.1 has rank R
 * at every bond (Lemma 4.2), so the products of Section 5.2 are applied straight from the
 * block form to dense tall matrices: Y = A Omega (Omega of Lemma 5.1 over the merged column
 * dims, Section 6.3, expanded densely), q power iterations (Alg. 5.4), Z = A^T Q = B^T, and the
 * small SVD of Alg. 5.1; without truncation this is TNrSVD in exact arithmetic. The tall
 * QRs are CholeskyQR2 in FP64 (a pass that breaks down is redone with the shift of shifted
 * CholeskyQR3). precision: TNR_FP64 or TNR_MIXED; both run the products in FP64 (on GB300 the
 * conversions an FP32 product of FP64 data needs cost more than the FP64 multiply-adds).
 * Outputs (device, column-major): U (nrows x k), S (k, descending), V (ncols x k).
 * ws: at least tnr_sparse_solve_workspace() bytes. Synchronises. Errors: TNR_EINVAL (dims
 * do not multiply to nrows / ncols, K > prod I or prod J), TNR_ERANGE (digits out of range,
 * sizes above 2^31), TNR_ENONFINITE (a Cholesky pivot that is not positive even after the
 * shift), TNR_ENOMEM. The workspace holds compact row and column lists of the nonzeros
 * (capacity R I_1 J_1 entries each).
 * ------------------------------------------------------------------------------------- */
int tnr_sparse_solve_workspace(int64_t nrows, int64_t ncols, int64_t R, int32_t d, const int64_t *I, const int64_t *J,
                               int32_t k, int32_t p, size_t *bytes);
int tnr_sparse_solve(int64_t nrows, int64_t ncols, int64_t R, const double *X, const uint8_t *digits, int32_t d,
                     const int64_t *I, const int64_t *J, int32_t k, int32_t p, int32_t q, uint64_t seed,
                     int32_t precision, double *U, double *S, double *V, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------------------
 * Differentiable TNrSVD (adjoint of Alg. 5.4 with Alg. 5.3 and Alg. 5.2), FP64 with fixed
 * ranks: tol = 0 (only exactly-zero singular values are dropped) and max_rank = K = k + p, so
 * the singular values S are a smooth function of A's cores where the singular values of every
 * step are simple. The paper has no adjoint; it is the reverse of its steps.
 * tnr_diff_forward: the same steps as tnr_solve (merge, Omega from `seed`, 2q+2 products,
 *   the two rounding sweeps of Section 5.4 and the site-1 factorisation per product, taken
 *   literally: no compression or no-truncation shortcuts) writing S (k doubles, device) and
 *   recording every step's factors in a tape (device memory allocated by the library on
 *   `stream`, stream-ordered). *tape receives an opaque handle. A's cores must stay unchanged
 *   until tnr_diff_backward. Synchronises. Errors: TNR_EINVAL, TNR_ENOMEM, TNR_ENONFINITE.
 * tnr_diff_backward: given dS (k doubles, device) = dL/dS, writes dL/dA into dA's cores
 *   (device buffers of A's shapes; dA->d, I, J, R as A). May run more than once per tape.
 *   Synchronises. TNR_ENONFINITE when a step's factor is singular (repeated or zero singular
 *   values, a singular R).
 * tnr_diff_free: releases a tape (null is ignored).
 * ------------------------------------------------------------------------------------- */
int tnr_diff_forward(const tnr_mpo *A, int32_t k, int32_t p, int32_t q, uint64_t seed, double *S, void **tape,
                     void *stream);
int tnr_diff_backward(void *tape, const double *dS, tnr_mpo *dA, void *stream);
void tnr_diff_free(void *tape, void *stream);

/* ---------------------------------------------------------------------------------------
 * Instrumentation (not part of the method): kernel launch counting and per-kernel-class
 * device time, measured with CUDA events recorded on the launching stream around each
 * launch while enabled. tnr_stats() synchronises and returns, for class `cls`, the number
 * of launches and the summed device milliseconds since the last reset; cls = -1 returns the
 * totals over all classes. tnr_stats_class_name() names a class (NULL past the last).
 * ------------------------------------------------------------------------------------- */
void tnr_stats_enable(int32_t class_mask); /* bit c: event-time class c */
void tnr_stats_reset(void);
int tnr_stats(int32_t cls, int64_t *launches, double *ms);
/* Algorithmic work recorded for class cls (or all, cls = -1) since the last reset: flops for
 * the FP64/tensor kernels (QR: dgeqrf + dorgqr counts; GEMM and products: 2 m n k), bytes
 * for the conversion kernels (24 B per nonzero read, the block values and digits written). */
int tnr_stats_work(int32_t cls, double *work);
const char *tnr_stats_class_name(int32_t cls);
/* CTAs per thread-block cluster that factor each bond of the exact compression (the cluster-
 * distributed column-pivoted QR of Section 5.4's rank-revealing step: 8 when the cooperative
 * launch with clusters is available, 1 when the one-CTA factorisation is used instead; 1 before
 * the first compression of the process). Instrumentation only. */
int tnr_compress_cluster_size(void);

const char *tnr_strerror(int status);
int tnr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TNRSVD_H */
