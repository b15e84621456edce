// Thread-block cluster primitives (one GPU): the cluster shape, the cluster barrier with
// release/acquire semantics, and stores into another CTA's shared memory (distributed shared
// memory, st.shared::cluster through a mapa-translated address).
#pragma once

#include <cstdint>

namespace tnr {

__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// barrier.cluster with release/acquire: shared-memory writes before it are visible to every CTA
// of the cluster after it. Executed by all threads, warp-converged.
__device__ __forceinline__ void cluster_sync_all() {
  __syncwarp();
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

// Address of `local` (a shared variable of this CTA) in the shared memory of cluster CTA `rank`.
__device__ __forceinline__ uint32_t dsmem_addr(const void *local, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void dsmem_st_f64(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

__device__ __forceinline__ void dsmem_st_s64(uint32_t a, long long v) {
  asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

__device__ __forceinline__ void dsmem_st_s32(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Stores v at `local` (an address of this CTA's shared memory) in every CTA of the cluster,
// this one included; the values are visible to each CTA after the next cluster_sync_all.
__device__ __forceinline__ void dsmem_put_all(double *local, double v, unsigned C) {
  for (unsigned rk = 0; rk < C; ++rk) dsmem_st_f64(dsmem_addr(local, rk), v);
}

}  // namespace tnr
