// One-sided (Hestenes) Jacobi iterations shared by the one-CTA SVD kernels.
//
// G (n x n, ld n) is rotated from the right until its columns are mutually orthogonal, and the
// rotations are accumulated into V (ld n): G_in V = G_out, G_out = U S. Column pairs follow a
// round-robin tournament, so the (n+1)/2 pairs of a round are disjoint. Each pair is handled by
// a group of g lanes (lanes = rows): GB300 issues FP64 at 1/64 of the FP32 rate, so one FP64
// warp instruction costs ~70 cycles of a sub-partition's FP64 pipe however many lanes are
// active, and the cheapest round packs several pairs into each warp (their rotation parameters
// then cost one instruction sequence per warp, not per pair) while using one warp per SM
// sub-partition (four), or all warps for large n. Column norms are recomputed at the start of
// each sweep and updated in between with the exact norms of the rotated pair. Columns whose norm
// is at the rounding level of the whole matrix (||g|| <= n eps ||G||_F) are numerically zero and
// are not rotated: rotating one against a large column only re-injects rounding error. A pair
// is skipped once |g_p^T g_q| <= tol ||g_p|| ||g_q||, tol = 16 eps sqrt(n).
#pragma once

#include <cfloat>
#include <cmath>

#include "dev_common.cuh"

namespace tnr {

// Pairs per warp for a matrix of n columns on a CTA of `warps` warps (a power of two <= 8).
__host__ __device__ inline int jacobi_pairs_per_warp(int n, int warps) {
  const int P = (n + 1) / 2;
  const int W = n > 64 ? warps : (warps < 4 ? warps : 4);
  int ppw = 1;
  while (ppw * W < P && ppw < 8) ppw <<= 1;
  return ppw;
}

// All threads of the CTA call this; nrm: n doubles of shared memory. Returns the sweep count.
static __device__ __noinline__ int jacobi_sweeps(double *G, double *V, int n, double *nrm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nthr = blockDim.x, nw = nthr >> 5;
  const int np = (n + 1) & ~1;
  const int ppw = jacobi_pairs_per_warp(n, nw);
  const int g = 32 / ppw, gi = lane / g, li = lane % g;
  const int pstride = nw * ppw;
  const double tolj = 16.0 * DBL_EPSILON * sqrt((double)(n > 4 ? n : 4));
  const double tol2 = tolj * tolj;
  __shared__ double s_fro2;
  __shared__ int s_rot2;
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    for (int j = threadIdx.x; j < n; j += nthr) {
      double s0 = 0.0, s1 = 0.0;
      int i = 0;
      for (; i + 1 < n; i += 2) {
        s0 = fma(G[i + n * j], G[i + n * j], s0);
        s1 = fma(G[i + 1 + n * j], G[i + 1 + n * j], s1);
      }
      if (i < n) s0 = fma(G[i + n * j], G[i + n * j], s0);
      nrm[j] = s0 + s1;
    }
    if (threadIdx.x == 0) s_rot2 = 0;
    __syncthreads();
    if (sweep == 0) {
      if (threadIdx.x == 0) {
        double f = 0.0;
        for (int j = 0; j < n; ++j) f += nrm[j];
        s_fro2 = f;
      }
      __syncthreads();
    }
    const double floor2 = (double)n * DBL_EPSILON * (double)n * DBL_EPSILON * s_fro2;
    for (int round = 0; round < np - 1; ++round) {
      for (int pbase = warp * ppw; pbase < np / 2; pbase += pstride) {
        const int pr = pbase + gi;
        int p = -1, q = -1;
        if (pr < np / 2) {
          if (pr == 0) {
            p = round;
            q = np - 1;
          } else {
            p = (round + pr) % (np - 1);
            q = (round - pr + (np - 1)) % (np - 1);
          }
          if (p > q) {
            const int x = p;
            p = q;
            q = x;
          }
        }
        bool act = p >= 0 && q < n;
        double al = 0.0, be = 0.0;
        if (act) {
          al = nrm[p];
          be = nrm[q];
          act = al > floor2 && be > floor2;
        }
        double ga = 0.0;
        if (act)
          for (int i = li; i < n; i += g) ga = fma(G[i + n * p], G[i + n * q], ga);
        for (int o = g >> 1; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o, g);
        double cs = 1.0, sn = 0.0;
        if (act) act = ga != 0.0 && ga * ga > tol2 * al * be && jacobi_rotation(al, be, ga, cs, sn);
        if (act) {
          double *gp = G + n * p, *gq = G + n * q, *vp = V + n * p, *vq = V + n * q;
          for (int i = li; i < n; i += g) {
            const double x = gp[i], y = gq[i];
            gp[i] = fma(-sn, y, cs * x);
            gq[i] = fma(sn, x, cs * y);
            const double xv = vp[i], yv = vq[i];
            vp[i] = fma(-sn, yv, cs * xv);
            vq[i] = fma(sn, xv, cs * yv);
          }
          if (li == 0) {
            const double c2 = cs * cs, s2 = sn * sn, cg = 2.0 * cs * sn * ga;
            nrm[p] = fma(c2, al, fma(s2, be, -cg));
            nrm[q] = fma(s2, al, fma(c2, be, cg));
            s_rot2 = 1;
          }
        }
      }
      __syncthreads();
    }
    const int rotated = s_rot2;
    __syncthreads();
    if (!rotated) break;
  }
  return sweep + 1;
}

}  // namespace tnr
