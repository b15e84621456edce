// One launch per truncated-SVD step of the right-to-left rounding sweep (Alg. 5.2 loop with the
// rounding of Section 5.4), for cores whose step fits one CTA's shared memory. The step itself
// (QR of the narrow side, no-truncation certificate, Jacobi SVD, truncation, outputs) is
// svd_step_cta in svd_step.cuh.
#include "svd_step.cuh"

namespace tnr {
namespace {

struct SvdStepArgs {
  const double *M;  // t x w, ld t
  int64_t t, w;
  const double *norm2;  // ||Y||_F^2 (device)
  double tol;
  int64_t dm1, max_rank;
  double *core_out;  // r x w, ld r (may alias M)
  double *US;        // t x r, ld t
  int64_t *r_out;
  int *status;
};

__global__ void __launch_bounds__(kStepThreads) k_svd_step(SvdStepArgs a) {
  extern __shared__ double sm[];
  const double delta2 = a.dm1 > 0 ? a.tol * a.tol * (*a.norm2) / (double)a.dm1 : 0.0;
  const int r = svd_step_cta(a.M, (int)a.t, (int)a.w, delta2, a.max_rank, a.core_out, a.US, sm, a.status);
  if (threadIdx.x == 0) *a.r_out = (int64_t)r;
}

}  // namespace

size_t svd_step_smem(int64_t t, int64_t w) { return sizeof(double) * (size_t)svd_step_work(t, w); }

int svd_step_small(cudaStream_t s, const double *M, int64_t t, int64_t w, const double *norm2, double tol,
                   int64_t dm1, int64_t max_rank, double *core_out, double *US, int64_t *r_dev) {
  const size_t smem = svd_step_smem(t, w);
  const int64_t n = t < w ? t : w;
  if (smem > 200 * 1024 || n > kStepMaxN) return TNR_EINVAL;
  SvdStepArgs a{M, t, w, norm2, tol, dm1, max_rank, core_out, US, r_dev, status_ptr()};
  TNR_TRY(ensure_dynamic_smem((const void *)k_svd_step, smem));
  LaunchScope ls(K_SVD, s);
  k_svd_step<<<1, kStepThreads, smem, s>>>(a);
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}

}  // namespace tnr
