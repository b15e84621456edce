// Column-pivoted Householder QR of a short wide matrix (m <= 64 rows, n columns) spread over the
// CTAs of one thread-block cluster: the rank-revealing factorisation of the exact compression
// (M_k^T = Q R P^T, stopped at the cutoff), with the same outputs as qr_tpc_cta.
//
// On one SM every pivot step is bound by the trailing update (about 2 m n FP64 FMAs through the
// SM's four FP64 pipes) plus the argmax -> reflector -> apply chain. Here CTA c of C owns the
// contiguous column block [c nl, (c + 1) nl), nl = ceil(n / C), so the update runs on C SMs. The
// exchange is push-only, so a pivot step has one cluster barrier and no remote loads:
//   1. at the end of step i-1 each of the four factorisation warps (one per SM sub-partition)
//      stores its best remaining column (norm key, index, and the column's rows i .. m-1) into
//      every CTA's receive buffers (st.shared::cluster; slots alternate by step parity);
//   2. barrier.cluster (release/acquire): all C x 4 candidates are in every CTA's shared memory;
//   3. every warp picks the same pivot p from them (largest remaining norm, ties to the lowest
//      column), so the cutoff test is decided identically in every CTA; a fifth warp forms the
//      Householder parameters from p's received column while the factorisation warps form the
//      partial dot products of their columns with it (they do not depend on the parameters), and
//      a named barrier of those five warps joins the two;
//   4. each factorisation warp applies the reflector to its columns (g lanes per column, a
//      group-local shuffle sum) and downdates the column norms (LAPACK dgeqp3 safeguard: recompute
//      once the downdate has lost half the digits), then posts its next candidate (1.).
// The cluster's control flow depends only on data every CTA holds identically, so all CTAs
// execute the same barriers.
// Outputs of qr_cluster_cta: L = R^T in the original column order (each CTA writes its own
// columns), the rank r to *r_out (CTA 0) and as the return value (every thread). Every CTA keeps
// the reflectors in its shared memory, so Q = H_0 .. H_{r-1} [I_r; 0] can be formed afterwards by
// qr_cluster_form_q (columns split over the cluster's warps) while other CTAs already use L. All
// threads of every CTA of the cluster call both.
#pragma once

#include <climits>

#include "cluster.cuh"
#include "dev_common.cuh"
#include "qr_tpc.cuh"

namespace tnr {

constexpr int kQrWarps = 4;        // factorisation warps per CTA: one per SM sub-partition
constexpr int kClusterMaxCtas = 8;  // portable cluster size limit

// Dynamic shared-memory bytes of qr_cluster_cta per CTA for an m x n matrix over C CTAs.
__host__ __device__ inline int64_t qr_cluster_bytes(int64_t m, int64_t n, int64_t C) {
  const int64_t nl = (n + C - 1) / C, nref = m < n ? m : n;
  return (int64_t)sizeof(double) * (m * nl + 3 * nl + m * nref + 2 * nref + kQrWarps * 64 + 2 * C * kQrWarps * 64) +
         (int64_t)sizeof(int) * nl;
}

// Lanes per column of the trailing update: the g minimising the FP64 warp instructions one
// sub-partition issues per step (column rounds per warp x (2 ceil(m / g) + log2 g + 4)).
__device__ __forceinline__ int qr_cluster_lg(int m, int nl) {
  int best = 0;
  long long best_cost = LLONG_MAX;
  for (int lg = 0; lg <= 5; ++lg) {
    const int g = 1 << lg, cpw = 32 >> lg;
    const int rounds = (nl + cpw - 1) / cpw;
    const long long per_warp = (rounds + kQrWarps - 1) / kQrWarps;
    const long long cost = per_warp * (2 * ((m + g - 1) / g) + lg + 4);
    if (cost < best_cost) {
      best_cost = cost;
      best = lg;
    }
  }
  return best;
}

// The shared-memory carve-up of one CTA (m x n over C CTAs).
struct QrClusterLayout {
  int nl, nref;
  double *A;     // m x nl row-major: A(t, jl) at t * nl + jl
  double *nrm;   // nl: squared norms below the active row
  double *thr;   // nl: 2^-26 x the squared norm at the last recompute
  double *dsum;  // nl: partial dot products of the current step (rows below the pivot row)
  double *V;     // m x nref: reflector i in column i (rows >= i)
  double *tau;   // nref
  double *bet;   // nref: R(i, p_i)
  double *vb;    // kQrWarps x 64: each warp's copy of the current reflector
  double *rcol;  // 2 x (C kQrWarps) x 64: received candidate columns, by step parity and slot
  int *step_of;  // nl: step a column was chosen
  __device__ QrClusterLayout(double *sm, int m, int n, int C) {
    nl = (n + C - 1) / C;
    nref = m < n ? m : n;
    A = sm;
    nrm = A + m * nl;
    thr = nrm + nl;
    dsum = thr + nl;
    V = dsum + nl;
    tau = V + m * nref;
    bet = tau + nref;
    vb = bet + nref;
    rcol = vb + kQrWarps * 64;
    step_of = reinterpret_cast<int *>(rcol + 2 * C * kQrWarps * 64);
  }
};

// Received candidates of the cluster (slot = CTA rank x kQrWarps + warp), by step parity.
struct QrClusterSlots {
  long long key[2][32];
  int idx[2][32];
  double fro[32];
};

// This warp's candidate for step s (its best remaining column: norm key and index, INT_MAX for
// none) with the column's rows s .. m-1, stored into every cluster CTA's receive buffers. All
// lanes call it (warp-converged) after the column's last update is visible to the warp.
static __device__ __forceinline__ void qr_cluster_post(const QrClusterLayout &lay, QrClusterSlots &sl, int m, int s,
                                                       long long key, int idx, int c0, unsigned C, unsigned me,
                                                       int warp, int lane) {
  const int slot = (int)me * kQrWarps + warp, b = s & 1;
  if (idx != INT_MAX) {
    const int jl = idx - c0, t0 = s + lane, t1 = s + lane + 32;
    const double x0 = t0 < m ? lay.A[t0 * lay.nl + jl] : 0.0;
    const double x1 = t1 < m ? lay.A[t1 * lay.nl + jl] : 0.0;
    double *dst = lay.rcol + (b * (int)C * kQrWarps + slot) * 64;
    for (unsigned rk = 0; rk < C; ++rk) {
      if (t0 < m) dsmem_st_f64(dsmem_addr(dst + t0, rk), x0);
      if (t1 < m) dsmem_st_f64(dsmem_addr(dst + t1, rk), x1);
    }
  }
  if (lane < (int)C) {
    dsmem_st_s64(dsmem_addr(&sl.key[b][slot], (unsigned)lane), key);
    dsmem_st_s32(dsmem_addr(&sl.idx[b][slot], (unsigned)lane), idx);
  }
}

// Warp-wide argmax of (key, column): largest key, ties to the lowest column; every lane gets it.
static __device__ __forceinline__ void warp_argmax(long long &k, int &j) {
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (ok > k || (ok == k && oj < j)) {
      k = ok;
      j = oj;
    }
  }
}

// Named barrier 1 among the factorisation warps and the parameter warp (kQrWarps + 1 warps).
__device__ __forceinline__ void qr_cluster_join() {
  asm volatile("bar.sync 1, %0;" ::"r"((kQrWarps + 1) * 32) : "memory");
}

static __device__ __noinline__ int qr_cluster_cta(const QrSmallArgs &a, double *sm) {
  const int m = (int)a.m, n = (int)a.n;
  const unsigned C = cluster_nctarank(), me = cluster_ctarank();
  const QrClusterLayout lay(sm, m, n, (int)C);
  const int nl = lay.nl, nref = lay.nref, c0 = (int)me * nl;
  double *A = lay.A, *nrm = lay.nrm, *thr = lay.thr, *V = lay.V, *tau = lay.tau, *bet = lay.bet, *vb = lay.vb;
  int *step_of = lay.step_of;
  __shared__ QrClusterSlots sl;
  __shared__ double s_hh[2];  // the current reflector's tau and scale
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lg = qr_cluster_lg(m, nl), g = 1 << lg, cpw = 32 >> lg, sub = lane & (g - 1);
  const int rounds = (nl + cpw - 1) / cpw;
  const unsigned gmask = g == 32 ? 0xffffffffu : ((1u << g) - 1u) << (lane & ~(g - 1));
  const int ncand = (int)C * kQrWarps;  // <= 32

  for (int idx = threadIdx.x; idx < m * nl; idx += blockDim.x) {
    const int t = idx / nl, jl = idx - t * nl, j = c0 + jl;
    // read through L2: the source may have been written by other CTAs of a cooperative kernel
    A[idx] = j < n ? __ldcg(a.trans_src ? a.src + (j + a.lds * t) : a.src + (t + a.lds * j)) : 0.0;
  }
  for (int jl = threadIdx.x; jl < nl; jl += blockDim.x) step_of[jl] = c0 + jl < n ? -1 : INT_MAX;
  __syncthreads();
  if (warp < kQrWarps) {  // initial norms, the Frobenius norm and the first candidates
    long long bk = -1;
    int bi = INT_MAX;
    double fro = 0.0;
    for (int rho = warp; rho < rounds; rho += kQrWarps) {
      const int jl = rho * cpw + (lane >> lg), j = c0 + jl;
      if (jl >= nl || j >= n) continue;  // uniform over the lane group
      double q = 0.0;
      for (int t = sub; t < m; t += g) q = fma(A[t * nl + jl], A[t * nl + jl], q);
      for (int o = 1; o < g; o <<= 1) q += __shfl_xor_sync(gmask, q, o);
      if (sub == 0) {
        nrm[jl] = q;
        thr[jl] = 0x1p-26 * q;
        fro += q;
        const long long key = __double_as_longlong(q);
        if (key > bk || (key == bk && j < bi)) {
          bk = key;
          bi = j;
        }
      }
    }
    warp_argmax(bk, bi);
    fro = dwarp_sum(fro);
    qr_cluster_post(lay, sl, m, 0, bk, bi, c0, C, me, warp, lane);
    if (lane < (int)C) dsmem_st_f64(dsmem_addr(&sl.fro[(int)me * kQrWarps + warp], (unsigned)lane), fro);
  }

  double cut2 = 0.0;
  int r = nref;
  for (int i = 0; i < nref; ++i) {
    cluster_sync_all();
    // every warp: the step's pivot from all candidates of the cluster (identical everywhere)
    const int b = i & 1;
    long long ck = lane < ncand ? sl.key[b][lane] : -1;
    int ci = lane < ncand ? sl.idx[b][lane] : INT_MAX;
    warp_argmax(ck, ci);
    if (i == 0)  // cutoff from the squared Frobenius norm, summed in a fixed lane order
      cut2 = a.cut_rel * a.cut_rel * dwarp_sum(lane < ncand ? sl.fro[lane] : 0.0);
    if (i > 0 && __longlong_as_double(ck) <= cut2) {
      r = i;
      break;
    }
    // Warp kQrWarps forms the reflector's parameters from p's received column (rows i .. m-1;
    // posted by the warp that updates column pl, slot own x kQrWarps + (pl / cpw) mod kQrWarps)
    // while the factorisation warps form the partial dot products d_j = sum_{t > i} x_t a_tj,
    // which do not depend on them; a named barrier joins the two. With v_i = 1, v_t = x_t scal:
    // w_j = tau (a_ij + scal d_j), a_ij <- a_ij - w_j, a_tj <- a_tj - (w_j scal) x_t.
    const int p = ci;
    const unsigned own = (unsigned)(p / nl);
    const int pl = p - (int)own * nl;
    const double *col = lay.rcol + (b * ncand + (int)own * kQrWarps + (pl / cpw) % kQrWarps) * 64;
    const int t0 = i + lane, t1 = i + lane + 32;
    if (warp > kQrWarps) continue;
    const double x0 = t0 < m ? col[t0] : 0.0;
    const double x1 = t1 < m ? col[t1] : 0.0;
    if (warp == kQrWarps) {
      const double alpha = __shfl_sync(0xffffffffu, x0, 0);
      const double sig = dwarp_sum(fma(x1, x1, lane > 0 ? x0 * x0 : 0.0));
      double tv = 0.0, beta = alpha, scal = 0.0;
      if (sig > 0.0) householder_params(alpha, sig, beta, tv, scal);
      if (lane == 0) {
        s_hh[0] = tv;
        s_hh[1] = scal;
        tau[i] = tv;
        bet[i] = beta;
        if (own == me) step_of[pl] = i;
      }
      qr_cluster_join();
      // the normalised reflector for the Q formation and the R output (off the critical path)
      if (t0 < m) V[i * m + t0] = lane == 0 ? 1.0 : x0 * scal;
      if (t1 < m) V[i * m + t1] = x1 * scal;
      continue;
    }
    double *v = vb + warp * 64;  // the raw column (rows > i are read)
    if (t0 < m) v[t0] = x0;
    if (t1 < m) v[t1] = x1;
    __syncwarp();
    for (int rho = warp; rho < rounds; rho += kQrWarps) {
      const int jl = rho * cpw + (lane >> lg), j = c0 + jl;
      if (jl >= nl || j == p || step_of[jl] >= 0) continue;  // uniform over the lane group
      const double *cj = A + jl;
      double dot = 0.0;
      for (int t = i + 1 + sub; t < m; t += g) dot = fma(v[t], cj[t * nl], dot);
      for (int o = 1; o < g; o <<= 1) dot += __shfl_xor_sync(gmask, dot, o);
      if (sub == 0) lay.dsum[jl] = dot;
    }
    qr_cluster_join();
    const double tv = s_hh[0], scal = s_hh[1];
    __syncwarp();  // each column's partial dot, stored by its group's first lane, is read by the group
    // apply to this warp's remaining columns; post the best remaining column for step i + 1
    long long bk = -1;
    int bi = INT_MAX;
    for (int rho = warp; rho < rounds; rho += kQrWarps) {
      const int jl = rho * cpw + (lane >> lg), j = c0 + jl;
      if (jl >= nl || j == p || step_of[jl] >= 0) continue;  // uniform over the lane group
      double *cj = A + jl;
      const double aij = cj[i * nl];
      double rij = aij;
      if (tv != 0.0) {
        const double w = tv * fma(scal, lay.dsum[jl], aij);
        const double ws = w * scal;
        for (int t = i + 1 + sub; t < m; t += g) cj[t * nl] = fma(-ws, v[t], cj[t * nl]);
        rij = aij - w;
        if (sub == 0) cj[i * nl] = rij;
      }
      double nn = fma(-rij, rij, nrm[jl]);
      if (nn <= thr[jl]) {  // cancelled (or negative): recompute from rows i+1 .. m-1
        double q = 0.0;
        for (int t = i + 1 + sub; t < m; t += g) q = fma(cj[t * nl], cj[t * nl], q);
        for (int o = 1; o < g; o <<= 1) q += __shfl_xor_sync(gmask, q, o);
        nn = q;
        if (sub == 0) thr[jl] = 0x1p-26 * q;
      }
      if (sub == 0) {
        nrm[jl] = nn;
        const long long key = __double_as_longlong(nn);
        if (key > bk || (key == bk && j < bi)) {
          bk = key;
          bi = j;
        }
      }
    }
    warp_argmax(bk, bi);
    __syncwarp();  // the candidate's updated rows, written by its lane group, are read by all lanes
    if (i + 1 < nref) qr_cluster_post(lay, sl, m, i + 1, bk, bi, c0, C, me, warp, lane);
  }
  // Every posted value was consumed before the loop ended (the last posts are read at the step
  // that stops), so no remote store is in flight and each CTA may reuse its shared memory. The
  // outputs read only this CTA's shared memory, but without a cutoff the last step's updates
  // may still be running in other warps: a CTA barrier orders them.
  __syncthreads();
  if (me == 0 && threadIdx.x == 0 && a.r_out) *a.r_out = r;
  // R^T (n x r, original column order) for this CTA's columns: a column chosen at step s keeps
  // rows < s, R(s, j) = beta_s and zeros below; the others hold row s after reflector s
  for (int idx = threadIdx.x; idx < r * nl; idx += blockDim.x) {
    const int s = idx / nl, jl = idx - s * nl, j = c0 + jl;
    if (j >= n) continue;
    const int so = step_of[jl];
    const double x = (so < 0 || s < so) ? A[s * nl + jl] : (s == so ? bet[so] : 0.0);
    if (a.trans_r)
      a.R[j + a.ldr * s] = x;
    else
      a.R[s + a.ldr * j] = x;
  }
  return r;
}

// Q (m x r) = H_0 .. H_{r-1} [I_r; 0] from the reflectors qr_cluster_cta left in every CTA's
// shared memory: column l by global warp l mod (C x warps), backward accumulation.
static __device__ __noinline__ void qr_cluster_form_q(const QrSmallArgs &a, double *sm, int r) {
  const int m = (int)a.m, n = (int)a.n;
  const unsigned C = cluster_nctarank(), me = cluster_ctarank();
  const QrClusterLayout lay(sm, m, n, (int)C);
  const double *V = lay.V, *tau = lay.tau;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldq = a.ldq > 0 ? (int)a.ldq : r;
  const int nwarps = (int)(blockDim.x >> 5);
  for (int l = (int)me * nwarps + warp; l < r; l += (int)C * nwarps) {
    const int u0 = lane, u1 = lane + 32;
    double q0 = u0 == l ? 1.0 : 0.0, q1 = u1 == l ? 1.0 : 0.0;
    for (int j = l; j >= 0; --j) {
      const double tj = tau[j];
      if (tj == 0.0) continue;
      const double w0 = u0 < j || u0 >= m ? 0.0 : V[j * m + u0];
      const double w1 = u1 < j || u1 >= m ? 0.0 : V[j * m + u1];
      const double w = dwarp_sum(fma(w0, q0, w1 * q1)) * tj;
      q0 = fma(-w, w0, q0);
      q1 = fma(-w, w1, q1);
    }
    if (a.trans_q) {
      if (u0 < m) a.Q[l + ldq * u0] = q0;
      if (u1 < m) a.Q[l + ldq * u1] = q1;
    } else {
      if (u0 < m) a.Q[u0 + ldq * l] = q0;
      if (u1 < m) a.Q[u1 + ldq * l] = q1;
    }
  }
}

}  // namespace tnr
