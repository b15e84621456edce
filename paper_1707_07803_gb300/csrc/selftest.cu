// Self-test of the bounded device waits: a wait that nothing will ever satisfy must end with
// TNR_ETIMEOUT in the device status word and leave the context usable. Two CTAs enter the grid
// barrier of the cooperative kernels (grid_sync.cuh); the second returns at once without arriving,
// so the first waits for an arrival that never comes until its poll cap runs out. Nothing faults or
// hangs: the wait is bounded by the caller's cap.
#include "grid_sync.cuh"

namespace tnr {
namespace {

__device__ unsigned g_selftest_bar[2];

__global__ void k_wait_never_satisfied(unsigned *bar, int *status, long long spin_cap) {
  if (blockIdx.x == 1) return;  // this CTA never arrives
  unsigned epoch = 0;
  grid_barrier(bar, status, epoch, spin_cap);
}

}  // namespace
}  // namespace tnr

using namespace tnr;

extern "C" int tnr_selftest_wait_timeout(int64_t spin_cap, void *stream) {
  if (spin_cap < 1 || spin_cap > kSpinCap) return TNR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned *bar = nullptr;
  TNR_CK(cudaGetSymbolAddress(reinterpret_cast<void **>(&bar), g_selftest_bar));
  TNR_TRY(reset_status(s));
  TNR_CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  k_wait_never_satisfied<<<2, 32, 0, s>>>(bar, status_ptr(), (long long)spin_cap);
  TNR_CK(cudaGetLastError());
  return read_status(s);  // TNR_ETIMEOUT when the bounded wait gave up, as it must
}
