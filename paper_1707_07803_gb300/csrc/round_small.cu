// Fused rounding sweeps for MPOs whose cores all fit in one CTA's shared memory.
//
// Section 5.4 integrates SVD-based rounding with the MPO-QR of Alg. 5.2: a left-to-right QR
// sweep (core k reshaped (R_k I_k J_k) x R_{k+1} = Q R, R absorbed into core k+1) followed by a
// right-to-left sweep that, per core, takes the truncated SVD of R_k x (I_k J_k R_{k+1}), keeps
// V^T as the new (right-orthogonal) core and absorbs U S into core k-1. When every core fits in
// shared memory the whole sequence is one launch: the cores are read once and written once, the
// ranks stay on the device, and each step's small dense factorisation is a device function run
// by the whole CTA, so there is no launch, host round trip or global-memory staging per bond.
// The site-1 step of Alg. 5.2/5.3 follows separately.
#include "round_small.cuh"

namespace tnr {
namespace {

__global__ void __launch_bounds__(kStepThreads) k_round_small(RoundSmallArgs a) {
  extern __shared__ double sm[];
  round_small_body(a, sm);
}

}  // namespace

// Runs both rounding sweeps of Y in one launch when they fit one CTA's shared memory; otherwise
// launches nothing and leaves *launched false. Ranks on exit go to R_dev (d + 1 values).
// certify: cores 1..d-1 are right-orthonormal, so the no-truncation certificate may skip the sweeps.
int round_small(cudaStream_t s, const tnr_mpo &Y, double tol, int64_t max_rank, bool certify, int64_t *R_dev,
                bool *launched) {
  *launched = false;
  RoundSmallLayout lay;
  int64_t phys[TNR_MAX_SITES];
  for (int k = 0; k < Y.d; ++k) phys[k] = Y.I[k] * Y.J[k];
  const size_t smem = round_small_layout(Y.R, phys, Y.d, &lay);
  if (smem == 0 || smem > kRoundSmallMaxSmem) return TNR_OK;
  RoundSmallArgs a;
  round_small_args(a, lay, Y.d, Y.core, Y.R, phys, certify, tol, max_rank, R_dev, status_ptr());
  TNR_TRY(ensure_dynamic_smem((const void *)k_round_small, smem));
  {
    LaunchScope ls(K_ROUND, s);
    k_round_small<<<1, kStepThreads, smem, s>>>(a);
  }
  TNR_CK(cudaGetLastError());
  *launched = true;
  return TNR_OK;
}

}  // namespace tnr
