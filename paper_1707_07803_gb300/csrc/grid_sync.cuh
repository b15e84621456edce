// Bounded grid-wide barrier for cooperative launches (all CTAs co-resident by construction).
// bar[0] counts arrivals, bar[1] is the generation; the last CTA to arrive resets the count and
// advances the generation. A waiter gives up after spin_cap polls (kSpinCap by default) and
// records TNR_ETIMEOUT instead of waiting forever. bar must be zeroed before the launch.
#pragma once

#include <cuda/atomic>

#include "tnr_internal.cuh"

namespace tnr {

static __device__ void grid_barrier(unsigned *bar, int *status, long long spin_cap = kSpinCap) {
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> count(bar[0]), gen(bar[1]);
    const unsigned my = gen.load(cuda::memory_order_acquire);
    __threadfence();
    if (count.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1) {
      count.store(0u, cuda::memory_order_relaxed);
      gen.fetch_add(1u, cuda::memory_order_release);
    } else {
      long long spins = 0;
      while (gen.load(cuda::memory_order_acquire) == my) {
        if (++spins > spin_cap) {
          set_status(status, TNR_ETIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace tnr
