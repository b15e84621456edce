// Bounded grid-wide barrier for cooperative launches (all CTAs co-resident by construction),
// counting arrivals: bar[0] counts every arrival of the launch (it is zeroed before the launch)
// and the e-th barrier completes when it reaches e x gridDim.x. Each CTA numbers its own barriers
// in `epoch` (the same sequence in every CTA), so an arrival is one release add and the wait one
// acquire poll: no generation word to read before arriving and no second atomic by the last
// arriver. A waiter gives up after spin_cap polls (kSpinCap by default) and records TNR_ETIMEOUT
// instead of waiting forever.
#pragma once

#include <cuda/atomic>

#include "tnr_internal.cuh"

namespace tnr {

static __device__ void grid_barrier(unsigned *bar, int *status, unsigned &epoch, long long spin_cap = kSpinCap) {
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> count(bar[0]);
    const unsigned target = epoch * gridDim.x;
    __threadfence();
    count.fetch_add(1u, cuda::memory_order_release);
    long long spins = 0;
    while (count.load(cuda::memory_order_acquire) < target) {
      if (++spins > spin_cap) {
        set_status(status, TNR_ETIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace tnr
