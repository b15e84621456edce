// The exact right-to-left compression of a product MPO (done before the rounding sweeps of
// Section 5.4) as one cooperative kernel.
//
// For k = d-1 .. 1 the compression factors M_k (t x w: core k with the already compressed right
// bond) as L Q_k by a column-pivoted QR of M_k^T that stops at the rounding-level cutoff; Q_k
// (orthonormal rows) becomes core k and L is absorbed into core k-1. Each bond needs the rank of
// the previous one, so the host-driven version reads a rank back and launches again for every
// bond. Here the whole sweep runs on the device: the first thread-block cluster factors M_k in
// shared memory (the cluster-distributed pivoted QR of qr_cluster.cuh: each of its CTAs owns a
// block of columns; without clusters, CTA 0 runs the thread-per-column QR of qr_tpc.cuh) while
// the other CTAs stage their blocks of rows of core k-1 in shared memory and wait at a grid
// barrier; then they multiply those rows by L (the absorb) while the cluster forms Q_k (only L is
// on the sweep's critical path), and the next bond starts after a second barrier.
// Ranks stay in device memory and are read back once at the end. A bond whose matrix does not
// fit the one-CTA QR (more than 64 rows, or beyond the shared-memory capacity) ends the kernel
// with the state of the host-driven sweep just before that bond, which the host then continues.
// The barriers spin with a bound (kSpinCap polls) and report TNR_ETIMEOUT instead of waiting
// forever; co-residency of all CTAs is guaranteed by the cooperative launch.
#include <algorithm>
#include <atomic>

#include "grid_sync.cuh"
#include "qr_cluster.cuh"
#include "qr_tpc.cuh"
#include "round_small.cuh"
#include "tnr_internal.cuh"

namespace tnr {
namespace {

struct CompressArgs {
  int d;
  double *core[TNR_MAX_SITES];
  int phys[TNR_MAX_SITES];   // I_k J_k
  int R[TNR_MAX_SITES + 1];  // ranks on entry
  double cut;
  double *L;             // t x r factor of the current bond (ld t)
  double *buf[2];        // absorbed cores (ping-pong), cap_buf doubles each
  int64_t cap_buf;
  int64_t qr_cap;        // shared-memory bytes available to the QR (per CTA)
  int64_t *R_out;        // ranks on exit (d + 1)
  unsigned *bar;         // [0] grid-barrier arrivals of the launch (zeroed before it)
  int *ctl;              // [0] first bond left to the host (0: none), [2] rounding done here
  int *status;
  // fused rounding (Section 5.4) after a complete compression, on CTA 0
  int fuse_round;
  double tol;
  int64_t max_rank;
  int64_t round_cap;     // dynamic shared-memory bytes of the launch (the rounding may use all)
  int64_t *R_round;      // ranks after the rounding (d + 1)
};

__global__ void __launch_bounds__(kSmallThreads) k_compress(CompressArgs a) {
  extern __shared__ double sm[];
  unsigned epoch = 0;  // grid barriers passed by this CTA
  const int d = a.d;
  const double *cur = a.core[d - 1];  // M_k (t x w, ld t)
  int rk1 = 1;                        // compressed rank of bond k+1
  const unsigned C = cluster_nctarank();  // CTAs of the factoring cluster (1: launched without)
  // the rounding has not run (yet): a later launch gated on this word must do nothing
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl[2] = 0;
  for (int k = d - 1; k >= 1; --k) {
    const int t = a.R[k], w = a.phys[k] * rk1;
    const bool fits = w <= 64 && (C > 1 ? qr_cluster_bytes(w, t, C) : qr_tpc_bytes(w, t)) <= a.qr_cap;
    if (!fits) {  // leave M_k in core k and bonds <= k to the host-driven sweep
      double *dst = a.core[k];
      if (cur != dst)
        for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)t * w;
             x += (int64_t)gridDim.x * blockDim.x)
          dst[x] = __ldcg(cur + x);
      if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl[0] = k;  // ranks of bonds > k are in R_out
      return;
    }
    int r_qr = 0;
    QrSmallArgs q;
    // absorbing CTAs (a cluster factors M_k): their block of rows of core k-1 staged in shared
    // memory while the cluster runs the QR (core k-1 is not written before its own bond)
    const unsigned first = C > 1 ? C : 0;  // CTAs that absorb: [first, gridDim.x)
    const int rows = a.R[k - 1] * a.phys[k - 1];
    const int nA = (int)gridDim.x - (int)first;
    const int rpb = (rows + nA - 1) / nA;
    const int arow0 = ((int)blockIdx.x - (int)first) * rpb;
    const int anrow = blockIdx.x >= first ? max(0, min(rpb, rows - arow0)) : 0;
    const bool pre = C > 1 && nA > 0 &&
                     ((int64_t)rpb * t + (int64_t)t * min(w, t)) * (int64_t)sizeof(double) <= a.round_cap;
    if (pre && blockIdx.x >= first) {
      const double *c0 = a.core[k - 1];
      for (int x = threadIdx.x; x < anrow * t; x += blockDim.x) {
        const int rr = x % anrow, j = x / anrow;
        sm[x] = __ldcg(c0 + arow0 + rr + (int64_t)rows * j);
      }
    }
    if (blockIdx.x < C) {  // M_k^T (w x t) = Q~ R~ P^T: core k <- Q~^T (r x w), L <- R~^T (t x r)
      q.src = cur;
      q.lds = t;
      q.m = w;
      q.n = t;
      q.trans_src = 1;
      q.pivot = 1;
      q.trans_q = 1;
      q.trans_r = 1;
      q.cut_rel = a.cut;
      q.Q = a.core[k];
      q.ldq = 0;
      q.R = a.L;
      q.ldr = t;
      q.r_out = a.R_out + k;
      if (C > 1)
        r_qr = qr_cluster_cta(q, sm);
      else
        qr_tpc_cta(q, sm);
    }
    grid_barrier(a.bar, a.status, epoch);
    // data written by other CTAs is read through L2 (__ldcg), never from a possibly stale L1 line;
    // the factoring cluster keeps its own rank, so its CTAs always agree on the next bond's shape
    // (and execute the same cluster barriers)
    const int r = (C > 1 && blockIdx.x < C) ? r_qr : (int)__ldcg(a.R_out + k);
    const double *Cc = a.core[k - 1];
    double *out = a.buf[k & 1];
    if (blockIdx.x < first) {
      qr_cluster_form_q(q, sm, r);  // core k <- Q~^T, beside the absorb
    } else if (pre) {
      // the staged rows times L (t x r, staged after them): eight lanes per output, each summing
      // the terms j = lane mod 8 in two chains, then a three-level shuffle sum (fixed order)
      const double *cs = sm;
      double *Ls = sm + (int64_t)anrow * t;
      for (int x = threadIdx.x; x < t * r; x += blockDim.x) Ls[x] = __ldcg(a.L + x);
      __syncthreads();
      const int part = threadIdx.x & 7, nout = anrow * r, ngroups = (int)(blockDim.x >> 3);
      // g0: the warp's first group, so the loop condition (and the shuffles) are warp-uniform
      for (int g = (int)(threadIdx.x >> 3), g0 = (int)(threadIdx.x >> 5) * 4; g0 < nout; g += ngroups, g0 += ngroups) {
        const bool live = g < nout;
        const int rr = live ? g % anrow : 0, c = live ? g / anrow : 0;
        double s0 = 0.0, s1 = 0.0;
        if (live) {
          const double *ci = cs + rr, *l = Ls + (int64_t)t * c;
          int j = part;
          for (; j + 8 < t; j += 16) {
            s0 = fma(ci[(int64_t)anrow * j], l[j], s0);
            s1 = fma(ci[(int64_t)anrow * (j + 8)], l[j + 8], s1);
          }
          if (j < t) s0 = fma(ci[(int64_t)anrow * j], l[j], s0);
        }
        double acc = s0 + s1;
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (live && part == 0) out[arow0 + rr + (int64_t)rows * c] = acc;
      }
    } else {
      // absorb: core k-1 (rows x t) L (t x r) -> buf (rows x r); L staged in shared memory (the
      // QR's buffer is free now), the core streamed from global memory
      double *Ls = sm;
      const bool staged = (int64_t)t * r * (int64_t)sizeof(double) <= a.round_cap;
      if (staged)
        for (int x = threadIdx.x; x < t * r; x += blockDim.x) Ls[x] = __ldcg(a.L + x);
      __syncthreads();
      // four lanes per output, lane `part` summing terms j = part mod 4 in four interleaved
      // chains (16 terms apart, so eight core loads are in flight per lane), combined in a fixed
      // order (deterministic); eight outputs per warp, consecutive rows (coalesced core reads)
      const int lane = threadIdx.x & 31, part = lane & 3;
      const int64_t nout = (int64_t)rows * r;
      const int64_t warps = ((int64_t)(gridDim.x - first) * blockDim.x) >> 5;
      for (int64_t g = ((int64_t)(blockIdx.x - first) * blockDim.x + threadIdx.x) >> 5; g * 8 < nout; g += warps) {
        const int64_t x = g * 8 + (lane >> 2);
        double acc = 0.0;
        if (x < nout) {
          const int i = (int)(x % rows), c = (int)(x / rows);
          const double *Ci = Cc + i;
          const double *l = staged ? Ls + t * c : a.L + (int64_t)t * c;
          double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
          int j = part;
#pragma unroll 2
          for (; j + 12 < t; j += 16) {
            const double c0 = Ci[(int64_t)rows * j], c1 = Ci[(int64_t)rows * (j + 4)];
            const double c2 = Ci[(int64_t)rows * (j + 8)], c3 = Ci[(int64_t)rows * (j + 12)];
            const double l0 = staged ? l[j] : __ldcg(l + j), l1 = staged ? l[j + 4] : __ldcg(l + j + 4);
            const double l2 = staged ? l[j + 8] : __ldcg(l + j + 8), l3 = staged ? l[j + 12] : __ldcg(l + j + 12);
            a0 = fma(c0, l0, a0);
            a1 = fma(c1, l1, a1);
            a2 = fma(c2, l2, a2);
            a3 = fma(c3, l3, a3);
          }
          for (; j < t; j += 4) a0 = fma(Ci[(int64_t)rows * j], staged ? l[j] : __ldcg(l + j), a0);
          acc = (a0 + a1) + (a2 + a3);
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (x < nout && part == 0) out[x] = acc;
      }
    }
    grid_barrier(a.bar, a.status, epoch);
    cur = out;
    rk1 = r;
  }
  // core 0 <- its absorbed form
  const int64_t n0 = (int64_t)a.phys[0] * rk1;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n0; x += (int64_t)gridDim.x * blockDim.x)
    a.core[0][x] = __ldcg(cur + x);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl[0] = 0;
    a.ctl[2] = 0;
    a.R_out[1] = rk1;
  }
  if (!a.fuse_round) return;
  // the certificate's first Gram G_1 = C_0^T C_0 (C_0: phys_0 x r_1, ld phys_0) spread over the
  // grid: CTA b sums a block of rows into partial b, in the ping-pong buffer not holding C_0
  const int p0 = a.phys[0];
  const int64_t g1_rows = (p0 + (int64_t)gridDim.x - 1) / gridDim.x;  // rows per CTA
  const bool g1_split = rk1 <= 16 && (int64_t)gridDim.x * rk1 * rk1 <= a.cap_buf &&
                        g1_rows * rk1 * (int64_t)sizeof(double) <= a.round_cap;
  double *g1p = a.buf[(cur == a.buf[0]) ? 1 : 0];
  if (g1_split) {
    const int rpb = (int)g1_rows, row0 = (int)blockIdx.x * rpb;
    const int nrow = max(0, min(rpb, p0 - row0));
    double *cs = sm;  // the block's rows, staged (nrow x rk1, ld nrow)
    for (int x = threadIdx.x; x < nrow * rk1; x += blockDim.x) {
      const int rr = x % nrow, c = x / nrow;
      cs[x] = __ldcg(cur + row0 + rr + (int64_t)p0 * c);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rk1 * rk1; e += blockDim.x) {
      const int i = e % rk1, j = e / rk1;
      double s0 = 0.0, s1 = 0.0;
      int rr = 0;
      for (; rr + 1 < nrow; rr += 2) {
        s0 = fma(cs[rr + nrow * i], cs[rr + nrow * j], s0);
        s1 = fma(cs[rr + 1 + nrow * i], cs[rr + 1 + nrow * j], s1);
      }
      if (rr < nrow) s0 = fma(cs[rr + nrow * i], cs[rr + nrow * j], s0);
      g1p[(int64_t)blockIdx.x * rk1 * rk1 + e] = s0 + s1;
    }
  }
  // every bond was compressed, so cores 1..d-1 are right-orthonormal: CTA 0 runs the rounding
  // sweeps (or their no-truncation certificate) on the compressed cores when they fit its
  // shared memory, leaving the final ranks in R_out
  grid_barrier(a.bar, a.status, epoch);
  if (blockIdx.x != 0) return;
  __shared__ int64_t s_R[TNR_MAX_SITES + 1], s_phys[TNR_MAX_SITES];
  __shared__ RoundSmallArgs s_args;
  __shared__ int s_fit;
  if (threadIdx.x == 0) {
    for (int k = 0; k <= d; ++k) s_R[k] = (k == 0 || k == d) ? 1 : __ldcg(a.R_out + k);
    for (int k = 0; k < d; ++k) s_phys[k] = a.phys[k];
    RoundSmallLayout lay;
    const size_t need = round_small_layout(s_R, s_phys, d, &lay);
    s_fit = need > 0 && (int64_t)need <= a.round_cap;
    if (s_fit) {
      round_small_args(s_args, lay, d, a.core, s_R, s_phys, true, a.tol, a.max_rank, a.R_round, a.status);
      if (g1_split) {
        s_args.g1_part = g1p;
        s_args.g1_parts = (int)gridDim.x;
      }
    }
    a.ctl[2] = s_fit;
  }
  __syncthreads();
  if (s_fit) round_small_body(s_args, sm);
}

}  // namespace

// Queues the compression of Y's bonds d-1 .. 1 on the device (no host synchronisation). With
// fuse_round, a complete compression is followed in the same launch by the rounding sweeps on
// CTA 0 (ctl[2] = 1 when they ran; R_round then holds the final ranks, d + 1 values). ctl[0] is
// the first bond left for the host-driven sweep (0: none); R_dev[k] the new rank of every bond the
// device finished. Scratch: L (maxbond x 64), two buffers of cap_buf doubles, ctl (>= 4 ints),
// bar (2). *launched = false when the shapes are outside the kernel's layout (nothing queued).
// Cluster size of the factoring cluster; whether the cooperative launch with clusters is
// available is decided at the first launch of the process (kept: -1 unknown, 0 refused, else C).
constexpr int kCompressCluster = 8;
// CTAs of the launch at most (whole clusters that fit): the absorb of each bond is bound by the
// FP64 instructions per SM, so it runs on every CTA outside the factoring cluster.
constexpr int kCompressGrid = 128;
static_assert(kCompressCluster * kQrWarps <= 32 && kCompressCluster <= kClusterMaxCtas,
              "one warp reads every candidate of the cluster; portable cluster size");
static_assert(kSmallThreads >= 32 * (kQrWarps + 1), "the cluster QR needs a parameter warp besides its factorisation warps");
static std::atomic<int> g_cluster_mode{-1};

int compress_cluster_size() { return g_cluster_mode.load() > 0 ? g_cluster_mode.load() : 1; }

int compress_launch(cudaStream_t s, const tnr_mpo &Y, double cut, double *L, double *buf0, double *buf1,
                    int64_t cap_buf, unsigned *bar, int *ctl, int64_t *R_dev, bool fuse_round, double tol,
                    int64_t max_rank, int64_t *R_round, bool *launched) {
  *launched = false;
  const int d = Y.d;
  if (d < 2) return TNR_OK;
  CompressArgs a;
  a.d = d;
  for (int k = 0; k < d; ++k) {
    const int64_t phys = Y.I[k] * Y.J[k];
    if (phys > (1 << 20) || Y.R[k] > (1 << 20) || Y.R[k] * phys * Y.R[k + 1] > cap_buf) return TNR_OK;
    a.core[k] = Y.core[k];
    a.phys[k] = (int)phys;
  }
  for (int k = 0; k <= d; ++k) a.R[k] = (int)Y.R[k];
  a.cut = cut;
  a.L = L;
  a.buf[0] = buf0;
  a.buf[1] = buf1;
  a.cap_buf = cap_buf;
  a.R_out = R_dev;
  a.bar = bar;
  a.ctl = ctl;
  a.status = status_ptr();
  a.fuse_round = fuse_round ? 1 : 0;
  a.tol = tol;
  a.max_rank = max_rank;
  a.R_round = R_round;
  int dev = 0, sms = 0;
  TNR_CK(cudaGetDevice(&dev));
  TNR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // clusters of kCompressCluster CTAs when available, else the one-CTA factorisation
  for (int C = g_cluster_mode.load() != 0 ? kCompressCluster : 1;; C = 1) {
    int64_t qr_need = 0;
    for (int k = 1; k < d; ++k) {
      const int64_t w = std::min<int64_t>(64, Y.I[k] * Y.J[k] * Y.R[k + 1]);
      qr_need = std::max(qr_need, C > 1 ? qr_cluster_bytes(w, Y.R[k], C) : qr_tpc_bytes(w, Y.R[k]));
    }
    const int64_t qr_cap = std::min<int64_t>(qr_need, 200 * 1024);
    const int64_t smem = fuse_round ? std::max<int64_t>(qr_cap, (int64_t)kRoundSmallMaxSmem) : qr_cap;
    a.qr_cap = qr_cap;
    a.round_cap = smem;
    TNR_TRY(ensure_dynamic_smem((const void *)k_compress, (size_t)smem));
    if (C > 1) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[2];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      at[1].id = cudaLaunchAttributeCooperative;
      at[1].val.cooperative = 1;
      cfg.gridDim = dim3(kCompressGrid);
      cfg.blockDim = dim3(kSmallThreads);
      cfg.dynamicSmemBytes = (size_t)smem;
      cfg.stream = s;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      // at least one cluster besides the factoring one: the other clusters' CTAs do the absorbs
      if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)k_compress, &cfg) != cudaSuccess || clusters < 2) {
        (void)cudaGetLastError();
        g_cluster_mode.store(0);
        continue;
      }
      cfg.gridDim = dim3((unsigned)(C * std::min(kCompressGrid / C, clusters)));
      cfg.numAttrs = 2;
      TNR_CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
      cudaError_t e;
      {
        LaunchScope ls(K_QR_PIV, s);
        e = cudaLaunchKernelEx(&cfg, k_compress, a);
      }
      if (e != cudaSuccess) {  // the cooperative launch with clusters was refused: one-CTA QR
        (void)cudaGetLastError();
        g_cluster_mode.store(0);
        continue;
      }
      g_cluster_mode.store(C);
      *launched = true;
      return TNR_OK;
    }
    int per_sm = 0;
    TNR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compress, kSmallThreads, (size_t)smem));
    if (per_sm < 1) return TNR_OK;
    const int blocks = std::min(kCompressGrid, sms * per_sm);
    TNR_CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    {
      LaunchScope ls(K_QR_PIV, s);
      void *args[] = {&a};
      TNR_CK(cudaLaunchCooperativeKernel((const void *)k_compress, dim3(blocks), dim3(kSmallThreads), args,
                                         (size_t)smem, s));
    }
    *launched = true;
    return TNR_OK;
  }
}

// Algorithmic flops of the bonds the device compressed (recorded once the ranks are known):
// r reflectors on w x t plus the explicit w x r Q, and the absorb 2 rows t r.
void compress_record_work(const tnr_mpo &Y, const int64_t *h, int first_host_bond) {
  double work = 0.0;
  int64_t rk1 = 1;
  for (int k = Y.d - 1; k > first_host_bond; --k) {
    const double t = (double)Y.R[k], w = (double)(Y.I[k] * Y.J[k] * rk1), r = (double)h[k];
    const double rows = (double)(Y.R[k - 1] * Y.I[k - 1] * Y.J[k - 1]);
    work += 4 * w * t * r - 2 * (w + t) * r * r + 4 * r * r * r / 3 + 2 * w * r * r - 2 * r * r * r / 3;
    work += 2 * rows * t * r;
    rk1 = h[k];
  }
  stats_work(K_QR_PIV, work);
}

}  // namespace tnr

extern "C" int tnr_compress_cluster_size(void) { return tnr::compress_cluster_size(); }
