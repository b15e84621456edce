// Tensor-core (tcgen05) contraction for the mixed-precision MPO products (Section 5.2).
//
// The site-1 product of A with Omega or Q is a dense GEMM (M = R2 * physical rows,
// N = K * S2, reduction over the shared physical index I1 or J1). It runs on the 5th-generation
// tensor cores: one elected thread issues tcgen05.mma.cta_group::1.kind::f16 with BF16 operands
// staged in shared memory (no-swizzle K-major core-matrix layout: 8 rows x 16 B per core matrix,
// LBO = 128 B between K-adjacent core matrices, SBO = (BK/8) * 128 B between 8-row groups) and
// FP32 accumulators in tensor memory (TMEM), read back with tcgen05.ld into registers for the
// FP64 epilogue store. Operands are FP64 in HBM and are rounded to BF16 while staging. With
// `split`, each operand x is written as hi + lo (hi = bf16(x), lo = bf16(x - hi)) and the tile
// product accumulates hi*hi + hi*lo + lo*hi: three BF16 MMAs per K-step give about 16 mantissa
// bits per product, FP32-class accuracy, at tensor-core speed.
//
// Synchronisation: the MMA completion is signalled by tcgen05.commit on an mbarrier; every
// wait on it is bounded (kSpinCap polls) and records TNR_ETIMEOUT on expiry, after which the
// CTA still frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "tnr_internal.cuh"

namespace tnr {
namespace {

constexpr int kTcM = 128;      // MMA M (cta_group::1)
constexpr int kTcBK = 64;      // K elements staged per stage (4 MMAs of K = 16)
// 8 warps: two per TMEM lane quadrant (tcgen05.ld reaches lanes 32 (warp mod 4) ..), splitting the
// epilogue's columns, and twice the threads of the operand conversions of one warp per quadrant
constexpr int kTcThreads = 256;

// index i -> (i % n1) * s1 + (i / n1) * s2
struct IdxMap {
  int64_t n1, s1, s2;
  __device__ __forceinline__ int64_t operator()(int64_t i) const {
    const unsigned ui = (unsigned)i, un = (unsigned)n1;  // all extents < 2^31
    return (int64_t)(ui % un) * s1 + (int64_t)(ui / un) * s2;
  }
};

struct TcArgs {
  const double *A;  // element (m, k) at A[amap(m) + k * a_ks]
  IdxMap amap;
  int64_t a_ks;
  const double *B;  // element (n, k) at B[bmap(n) + k * b_ks]
  IdxMap bmap;
  int64_t b_ks;
  double *C;  // element (m, n) at C[crow(m) + ccol(n)]
  IdxMap crow, ccol;
  int64_t M, N, K;
  int BN;        // N tile (multiple of 16, <= 256)
  int tmem_cols; // power of two >= max(32, BN)
  int split;
  int *status;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// byte offset of element (r, k) in a K-major no-swizzle tile with BK columns
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
  return (uint32_t)((r >> 3) * (kTcBK / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *status) {
  for (long long it = 0; it < kSpinCap; ++it) {
    uint32_t ok = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  set_status(status, TNR_ETIMEOUT);
  return false;
}

__global__ void __launch_bounds__(kTcThreads) k_tc_gemm(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_abort;
  __shared__ int64_t s_arow[kTcM], s_bcol[256], s_crow[kTcM], s_ccol[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kTcM;
  const int64_t n0 = (int64_t)blockIdx.y * a.BN;
  const int parts = a.split ? 2 : 1;
  // stage layout: A_hi, A_lo, B_hi, B_lo (bf16 tiles)
  const uint32_t a_bytes = kTcM * kTcBK * 2, b_bytes = (uint32_t)a.BN * kTcBK * 2;
  unsigned char *sA[2] = {tsm, tsm + a_bytes};
  unsigned char *sB[2] = {tsm + parts * a_bytes, tsm + parts * a_bytes + b_bytes};

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  // per-row / per-column base offsets of this tile (one index split each)
  for (int i = threadIdx.x; i < kTcM; i += kTcThreads) {
    const int64_t gm = m0 + i;
    s_arow[i] = gm < a.M ? a.amap(gm) : -1;
    s_crow[i] = gm < a.M ? a.crow(gm) : -1;
  }
  for (int i = threadIdx.x; i < a.BN; i += kTcThreads) {
    const int64_t gn = n0 + i;
    s_bcol[i] = gn < a.N ? a.bmap(gn) : -1;
    s_ccol[i] = gn < a.N ? a.ccol(gn) : -1;
  }
  __syncthreads();

  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.BN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint32_t sbo = (kTcBK / 8) * 128, lbo = 128;
  uint32_t phase = 0;
  const int64_t nkb = (a.K + kTcBK - 1) / kTcBK;
  for (int64_t kb = 0; kb < nkb; ++kb) {
    const int64_t k0 = kb * kTcBK;
    // stage A (128 x BK) and B (BN x BK), FP64 -> BF16 (hi, lo). One FP64-pipe conversion per
    // element (double -> float); the hi/lo split is done in FP32 (hi + lo carries 16 significant
    // bits, far inside FP32's 24). Loads are issued four at a time before any conversion.
    {
      constexpr int U = 4;
      const int na = kTcM * kTcBK;
      for (int base_idx = threadIdx.x; base_idx < na; base_idx += kTcThreads * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base_idx + u * kTcThreads;
          x[u] = 0.0;
          if (idx < na) {
            const int r = a.a_ks == 1 ? idx / kTcBK : idx % kTcM;
            const int k = a.a_ks == 1 ? idx % kTcBK : idx / kTcM;
            const int64_t gk = k0 + k, base = s_arow[r];
            if (base >= 0 && gk < a.K) x[u] = a.A[base + gk * a.a_ks];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base_idx + u * kTcThreads;
          if (idx >= na) continue;
          const int r = a.a_ks == 1 ? idx / kTcBK : idx % kTcM;
          const int k = a.a_ks == 1 ? idx % kTcBK : idx / kTcM;
          const float f = (float)x[u];
          const __nv_bfloat16 hi = __float2bfloat16(f);
          *reinterpret_cast<__nv_bfloat16 *>(sA[0] + kmajor_off(r, k)) = hi;
          if (a.split) *reinterpret_cast<__nv_bfloat16 *>(sA[1] + kmajor_off(r, k)) = __float2bfloat16(f - __bfloat162float(hi));
        }
      }
      const int nb = a.BN * kTcBK;
      for (int base_idx = threadIdx.x; base_idx < nb; base_idx += kTcThreads * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base_idx + u * kTcThreads;
          x[u] = 0.0;
          if (idx < nb) {
            const int r = a.b_ks == 1 ? idx / kTcBK : idx % a.BN;
            const int k = a.b_ks == 1 ? idx % kTcBK : idx / a.BN;
            const int64_t gk = k0 + k, base = s_bcol[r];
            if (base >= 0 && gk < a.K) x[u] = a.B[base + gk * a.b_ks];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base_idx + u * kTcThreads;
          if (idx >= nb) continue;
          const int r = a.b_ks == 1 ? idx / kTcBK : idx % a.BN;
          const int k = a.b_ks == 1 ? idx % kTcBK : idx / a.BN;
          const float f = (float)x[u];
          const __nv_bfloat16 hi = __float2bfloat16(f);
          *reinterpret_cast<__nv_bfloat16 *>(sB[0] + kmajor_off(r, k)) = hi;
          if (a.split) *reinterpret_cast<__nv_bfloat16 *>(sB[1] + kmajor_off(r, k)) = __float2bfloat16(f - __bfloat162float(hi));
        }
      }
    }
    // make generic-proxy smem writes visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kk = 0; kk < kTcBK; kk += 16) {
        const uint32_t koff = (uint32_t)(kk / 8) * 128;
        // (A part, B part) pairs: hi*hi, then hi*lo and lo*hi when split
        const int npairs = a.split ? 3 : 1;
        for (int pr = 0; pr < npairs; ++pr) {
          const int ap = pr == 2 ? 1 : 0, bp = pr == 1 ? 1 : 0;
          const uint64_t ad = make_desc(smem_u32(sA[ap]) + koff, lbo, sbo);
          const uint64_t bd = make_desc(smem_u32(sB[bp]) + koff, lbo, sbo);
          const uint32_t acc = (kb > 0 || kk > 0 || pr > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    // wait for the MMAs before the next stage overwrites the tiles (and before the epilogue)
    if (!mbar_wait(smem_u32(&mbar), phase, a.status)) {
      if (threadIdx.x == 0) s_abort = 1;
    }
    phase ^= 1;
    __syncthreads();
    if (s_abort) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_abort) {
    // epilogue: warps w and w + 4 own TMEM lanes 32w..32w+31 = tile rows, alternate 8-column groups
    const int quad = warp & 3, nh = kTcThreads / 128;
    const int64_t rowoff = s_crow[quad * 32 + lane];
    for (int c0 = (warp >> 2) * 8; c0 < a.BN; c0 += 8 * nh) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (rowoff >= 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t co = s_ccol[c0 + j];
          if (co >= 0) a.C[rowoff + co] = (double)__uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// TMA-staged variant. Each K-stage of kTmaBK columns is fetched as two 3-D FP64 boxes by the
// tensor-memory accelerator (cp.async.bulk.tensor, completion counted on an mbarrier with
// expect_tx; out-of-range parts of a box arrive as zeros), then all threads round the FP64 tiles
// in shared memory to BF16 (hi, lo) in the K-major core-matrix layout the MMAs read, and one
// elected thread issues the tcgen05.mma sequence as in k_tc_gemm. Used when the operands satisfy
// the TMA rules (16-byte aligned bases, strides multiple of 16 bytes, even x coordinates) and the
// tiles are whole boxes: 128 rows of A = (bx rows) x (by groups), N = Kx S2 <= 256, N % 16 == 0.
constexpr int kTmaBK = 32;

struct TmaArgs {
  int trans;     // A box: (rows0, K, groups) for trans 0, (K, rows0, groups) for trans 1
  int box_r0;    // rows of A per group in the box (I or J part), box_r0 * box_g = 128
  int rows0;     // the full extent of that row index (I for trans 0, J for trans 1)
  int64_t M, N, K;
  int BN;        // = N
  int tmem_cols;
  int split;
  double *C;
  IdxMap crow, ccol;
  int *status;
};

__device__ __forceinline__ uint32_t kmajor_off32(int r, int k) {
  return (uint32_t)((r >> 3) * (kTmaBK / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(kTcThreads) k_tc_gemm_tma(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB, TmaArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar, tbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_abort;
  __shared__ int64_t s_crow[kTcM], s_ccol[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kTcM;
  const int parts = a.split ? 2 : 1;
  // FP64 boxes (1024-aligned), then the BF16 tiles: A_hi, A_lo, B_hi, B_lo
  const uint32_t fa_bytes = kTcM * kTmaBK * 8, fb_bytes = (uint32_t)a.BN * kTmaBK * 8;
  const uint32_t a_bytes = kTcM * kTmaBK * 2, b_bytes = (uint32_t)a.BN * kTmaBK * 2;
  const double *fA = reinterpret_cast<const double *>(tsm);
  const double *fB = reinterpret_cast<const double *>(tsm + fa_bytes);
  unsigned char *bf = tsm + fa_bytes + ((fb_bytes + 1023) & ~1023u);
  unsigned char *sA[2] = {bf, bf + a_bytes};
  unsigned char *sB[2] = {bf + parts * a_bytes, bf + parts * a_bytes + b_bytes};

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  for (int i = threadIdx.x; i < kTcM; i += kTcThreads) s_crow[i] = m0 + i < a.M ? a.crow(m0 + i) : -1;
  for (int i = threadIdx.x; i < a.BN; i += kTcThreads) s_ccol[i] = i < a.N ? a.ccol(i) : -1;
  // box coordinates of this CTA's 128 rows: (row within the group, group)
  const int r0c = (int)(m0 % a.rows0), g0c = (int)(m0 / a.rows0);
  __syncthreads();

  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.BN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint32_t sbo = (kTmaBK / 8) * 128, lbo = 128;
  uint32_t phase = 0, tphase = 0;
  const int64_t nkb = (a.K + kTmaBK - 1) / kTmaBK;
  for (int64_t kb = 0; kb < nkb; ++kb) {
    const int k0 = (int)(kb * kTmaBK);
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&tbar)),
                   "r"(fa_bytes + fb_bytes)
                   : "memory");
      if (a.trans == 0)
        tma_load_3d(smem_u32(fA), &tmA, r0c, k0, g0c, smem_u32(&tbar));
      else
        tma_load_3d(smem_u32(fA), &tmA, k0, r0c, g0c, smem_u32(&tbar));
      tma_load_3d(smem_u32(fB), &tmB, k0, 0, 0, smem_u32(&tbar));
    }
    if (!mbar_wait(smem_u32(&tbar), tphase, a.status) && threadIdx.x == 0) s_abort = 1;
    tphase ^= 1;
    __syncthreads();
    if (s_abort) break;
    // FP64 boxes -> BF16 (hi, lo) K-major tiles; one FP64-pipe conversion per element
    for (int idx = threadIdx.x; idx < kTcM * kTmaBK; idx += kTcThreads) {
      int r, k;
      if (a.trans == 0) {  // box [group][k][row0]
        const int i = idx % a.box_r0, rest = idx / a.box_r0;
        k = rest % kTmaBK;
        r = i + a.box_r0 * (rest / kTmaBK);
      } else {  // box [group][row0][k]
        k = idx % kTmaBK;
        r = idx / kTmaBK;
      }
      const float f = (float)fA[idx];
      const __nv_bfloat16 hi = __float2bfloat16(f);
      *reinterpret_cast<__nv_bfloat16 *>(sA[0] + kmajor_off32(r, k)) = hi;
      if (a.split) *reinterpret_cast<__nv_bfloat16 *>(sA[1] + kmajor_off32(r, k)) = __float2bfloat16(f - __bfloat162float(hi));
    }
    for (int idx = threadIdx.x; idx < a.BN * kTmaBK; idx += kTcThreads) {  // box [s2][c][k]
      const int k = idx % kTmaBK, n = idx / kTmaBK;
      const float f = (float)fB[idx];
      const __nv_bfloat16 hi = __float2bfloat16(f);
      *reinterpret_cast<__nv_bfloat16 *>(sB[0] + kmajor_off32(n, k)) = hi;
      if (a.split) *reinterpret_cast<__nv_bfloat16 *>(sB[1] + kmajor_off32(n, k)) = __float2bfloat16(f - __bfloat162float(hi));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kk = 0; kk < kTmaBK; kk += 16) {
        const uint32_t koff = (uint32_t)(kk / 8) * 128;
        const int npairs = a.split ? 3 : 1;
        for (int pr = 0; pr < npairs; ++pr) {
          const int ap = pr == 2 ? 1 : 0, bp = pr == 1 ? 1 : 0;
          const uint64_t ad = make_desc(smem_u32(sA[ap]) + koff, lbo, sbo);
          const uint64_t bd = make_desc(smem_u32(sB[bp]) + koff, lbo, sbo);
          const uint32_t acc = (kb > 0 || kk > 0 || pr > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    // the MMAs must finish before the next stage rewrites the BF16 tiles
    if (!mbar_wait(smem_u32(&mbar), phase, a.status) && threadIdx.x == 0) s_abort = 1;
    phase ^= 1;
    __syncthreads();
    if (s_abort) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_abort) {
    const int quad = warp & 3, nh = kTcThreads / 128;  // as in k_tc_gemm
    const int64_t rowoff = s_crow[quad * 32 + lane];
    for (int c0 = (warp >> 2) * 8; c0 < a.BN; c0 += 8 * nh) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (rowoff >= 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t co = s_ccol[c0 + j];
          if (co >= 0) a.C[rowoff + co] = (double)__uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D FP64 tensor map (dims d0 fastest, byte strides s1, s2) with the given box; false when the
// encoder refuses it or is unavailable.
bool encode_3d(CUtensorMap *map, const double *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1, uint64_t s2,
               uint32_t b0, uint32_t b1, uint32_t b2) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {s1, s2};
  const cuuint32_t box[3] = {b0, b1, b2};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The TMA-staged launch when the shapes allow it (*done = false otherwise, nothing queued).
int contract_site1_tma(cudaStream_t s, const double *A, int64_t I, int64_t J, int64_t R2, const double *X, int64_t Kx,
                       int64_t S2, int trans, double *Y, bool split, bool *done) {
  *done = false;
  const int64_t Xo = trans ? J : I, Ny = trans ? I : J;
  const int64_t M = Xo * R2, N = Kx * S2;
  const int64_t rows0 = Xo;  // the row index inside a group (i for trans 0, j for trans 1)
  if (N % 16 != 0 || N < 16 || N > 256 || Kx > 256 || S2 > 256) return TNR_OK;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(X) & 15)) return TNR_OK;
  if ((I * 8) % 16 || (Ny * 8) % 16 || I * J * R2 >= (int64_t)1 << 31 || Ny * N >= (int64_t)1 << 31) return TNR_OK;
  int64_t box_r0, box_g;
  if (rows0 <= kTcM && kTcM % rows0 == 0) {
    box_r0 = rows0;
    box_g = kTcM / rows0;
  } else if (rows0 % kTcM == 0) {
    box_r0 = kTcM;
    box_g = 1;
  } else {
    return TNR_OK;
  }
  if (box_r0 % 2 || box_g > 256 || R2 > ((int64_t)1 << 31)) return TNR_OK;  // even x coordinates (trans 0)
  CUtensorMap mA, mB;
  // A(i, j, r2) at i + I j + I J r2: dims (I, J, R2)
  const bool okA = trans == 0 ? encode_3d(&mA, A, I, J, R2, I * 8, I * J * 8, (uint32_t)box_r0, kTmaBK, (uint32_t)box_g)
                              : encode_3d(&mA, A, I, J, R2, I * 8, I * J * 8, kTmaBK, (uint32_t)box_r0, (uint32_t)box_g);
  // X(y, c, s2) at y + Ny (c + Kx s2): dims (Ny, Kx, S2), one box for all N columns
  const bool okB = encode_3d(&mB, X, Ny, Kx, S2, Ny * 8, Ny * Kx * 8, kTmaBK, (uint32_t)Kx, (uint32_t)S2);
  if (!okA || !okB) return TNR_OK;
  TmaArgs a;
  a.trans = trans;
  a.box_r0 = (int)box_r0;
  a.rows0 = (int)rows0;
  a.M = M;
  a.N = N;
  a.K = Ny;
  a.BN = (int)N;
  int tc = 32;
  while (tc < a.BN) tc <<= 1;
  a.tmem_cols = tc;
  a.split = split ? 1 : 0;
  a.C = Y;  // Y(0, xo, c, r2 + R2 s2) at xo + Xo (c + Kx (r2 + R2 s2))
  a.crow = {Xo, 1, Xo * Kx};
  a.ccol = {Kx, Xo, Xo * Kx * R2};
  a.status = status_ptr();
  const int parts = split ? 2 : 1;
  const size_t fb = ((size_t)N * kTmaBK * 8 + 1023) & ~size_t(1023);
  const size_t smem = (size_t)kTcM * kTmaBK * 8 + fb + (size_t)parts * (kTcM * kTmaBK * 2 + (size_t)N * kTmaBK * 2) + 1024;
  TNR_TRY(ensure_dynamic_smem((const void *)k_tc_gemm_tma, smem));
  const dim3 grid((unsigned)cdiv(M, kTcM), 1);
  stats_work(K_CONTRACT_TC, 2.0 * (double)M * (double)N * (double)Ny * (split ? 3.0 : 1.0));
  {
    LaunchScope ls(K_CONTRACT_TC, s);
    k_tc_gemm_tma<<<grid, kTcThreads, smem, s>>>(mA, mB, a);
  }
  TNR_CK(cudaGetLastError());
  *done = true;
  return TNR_OK;
}

}  // namespace

// Site-level tensor-core product for a site with R = S = 1 boundary bonds on the left (site 1):
// Y(0, xo, c, (r2, s2)) = sum_y A(0, i, j, r2) X(0, y, c, s2), (xo, y) = (i, j) or (j, i).
int contract_site1_tc(cudaStream_t s, const double *A, int64_t I, int64_t J, int64_t R2, const double *X, int64_t Kx,
                      int64_t S2, int trans, double *Y, bool split) {
  bool done = false;
  TNR_TRY(contract_site1_tma(s, A, I, J, R2, X, Kx, S2, trans, Y, split, &done));
  if (done) return TNR_OK;
  TcArgs a;
  const int64_t Xo = trans ? J : I, Ny = trans ? I : J;
  a.A = A;
  if (!trans) {  // rows (i, r2), k = j: A(i, j, r2) at i + I j + I J r2
    a.amap = {I, 1, I * J};
    a.a_ks = I;
  } else {  // rows (j, r2), k = i: A(i, j, r2) at i + I j + I J r2
    a.amap = {J, I, I * J};
    a.a_ks = 1;
  }
  a.B = X;  // X(0, y, c, s2) at y + Ny (c + Kx s2): cols (c, s2), k = y
  a.bmap = {Kx, Ny, Ny * Kx};
  a.b_ks = 1;
  a.C = Y;  // Y(0, xo, c, r2 + R2 s2) at xo + Xo (c + Kx (r2 + R2 s2))
  a.crow = {Xo, 1, Xo * Kx};
  a.ccol = {Kx, Xo, Xo * Kx * R2};
  a.M = Xo * R2;
  a.N = Kx * S2;
  a.K = Ny;
  int64_t bn = ((a.N + 15) / 16) * 16;
  if (bn > 256) bn = 256;
  a.BN = (int)bn;
  int tc = 32;
  while (tc < a.BN) tc <<= 1;
  a.tmem_cols = tc;
  a.split = split ? 1 : 0;
  a.status = status_ptr();
  const int parts = split ? 2 : 1;
  const size_t smem = (size_t)parts * (kTcM * kTcBK * 2 + (size_t)a.BN * kTcBK * 2) + 1024;
  TNR_TRY(ensure_dynamic_smem((const void *)k_tc_gemm, smem));
  dim3 grid((unsigned)cdiv(a.M, kTcM), (unsigned)cdiv(a.N, a.BN));
  stats_work(K_CONTRACT_TC, 2.0 * (double)a.M * (double)a.N * (double)a.K * (split ? 3.0 : 1.0));
  LaunchScope ls(K_CONTRACT_TC, s);
  k_tc_gemm<<<grid, kTcThreads, smem, s>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    fprintf(stderr, "libtnrsvd: k_tc_gemm launch M=%lld N=%lld K=%lld BN=%d grid=%ux%u smem=%zu\n", (long long)a.M,
            (long long)a.N, (long long)a.K, a.BN, grid.x, grid.y, smem);
  return check_cuda_at(e, __FILE__, __LINE__);
}

}  // namespace tnr
