// One-sided (Hestenes) Jacobi iterations shared by the one-CTA SVD kernels.
//
// G (n x n, leading dimension ld) is rotated from the right until its columns are mutually
// orthogonal, and the rotations are accumulated into V (same layout): G_in V = G_out, G_out = U S. Column pairs follow a
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
// The sweeps are written once for FP32 and FP64 (plus a one-warp-per-pair FP32 variant for
// n <= 32); jacobi_sweeps_mixed runs them in FP32 first and finishes in FP64 (see there), which is
// what the SVD kernels call, optionally by the matrix-product refinement instead of FP64 sweeps.
#pragma once

#include <cfloat>
#include <cmath>

#include "cluster.cuh"
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

// FP32 rotation of the preconditioning pass (same formulas as jacobi_rotation, in FP32).
__device__ __forceinline__ bool jacobi_rotation_f32(float al, float be, float ga, float &cs, float &sn) {
  const float z = (be - al) / (2.0f * ga);
  if (!isfinite(z)) return false;
  const float t = copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f)));
  if (t == 0.0f || !isfinite(t)) return false;
  cs = rsqrtf(fmaf(t, t, 1.0f));
  sn = cs * t;
  return true;
}
__device__ __forceinline__ bool jacobi_rot(double al, double be, double ga, double &cs, double &sn) {
  return jacobi_rotation(al, be, ga, cs, sn);
}
__device__ __forceinline__ bool jacobi_rot(float al, float be, float ga, float &cs, float &sn) {
  return jacobi_rotation_f32(al, be, ga, cs, sn);
}
template <typename T>
struct JacobiEps;
template <>
struct JacobiEps<double> {
  static __device__ __forceinline__ double eps() { return DBL_EPSILON; }
};
template <>
struct JacobiEps<float> {
  static __device__ __forceinline__ float eps() { return FLT_EPSILON; }
};

// All threads of the CTA call this; G and V are n x n with leading dimension ld (n + 1 keeps the
// columns a warp rotates at once in different shared-memory banks); nrm: n values of shared
// memory. Returns the sweep count.
template <typename T>
static __device__ __noinline__ int jacobi_sweeps_t(T *G, T *V, int n, int ld, T *nrm, int max_sweeps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nthr = blockDim.x, nw = nthr >> 5;
  const int np = (n + 1) & ~1;
  const int ppw = jacobi_pairs_per_warp(n, nw);
  const int g = 32 / ppw, gi = lane / g, li = lane % g;
  const int pstride = nw * ppw;
  const T eps = JacobiEps<T>::eps();
  const T tolj = (T)16 * eps * (T)sqrt((double)(n > 4 ? n : 4));
  const T tol2 = tolj * tolj;
  __shared__ T s_fro2;
  __shared__ int s_rot2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = threadIdx.x; j < n; j += nthr) {
      T s0 = 0, s1 = 0;
      int i = 0;
      for (; i + 1 < n; i += 2) {
        s0 = fma(G[i + ld * j], G[i + ld * j], s0);
        s1 = fma(G[i + 1 + ld * j], G[i + 1 + ld * j], s1);
      }
      if (i < n) s0 = fma(G[i + ld * j], G[i + ld * j], s0);
      nrm[j] = s0 + s1;
    }
    if (threadIdx.x == 0) s_rot2 = 0;
    __syncthreads();
    if (sweep == 0) {
      if (threadIdx.x == 0) {
        T f = 0;
        for (int j = 0; j < n; ++j) f += nrm[j];
        s_fro2 = f;
      }
      __syncthreads();
    }
    const T floor2 = (T)n * eps * (T)n * eps * s_fro2;
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
        T al = 0, be = 0;
        if (act) {
          al = nrm[p];
          be = nrm[q];
          act = al > floor2 && be > floor2;
        }
        T ga = 0;
        if (act) {  // four rows in flight per lane (operands may sit in global memory)
          const T *gp = G + ld * p, *gq = G + ld * q;
          T a1 = 0, a2 = 0, a3 = 0;
          int i = li;
          for (; i + 3 * g < n; i += 4 * g) {
            const T x0 = gp[i], x1 = gp[i + g], x2 = gp[i + 2 * g], x3 = gp[i + 3 * g];
            const T y0 = gq[i], y1 = gq[i + g], y2 = gq[i + 2 * g], y3 = gq[i + 3 * g];
            ga = fma(x0, y0, ga);
            a1 = fma(x1, y1, a1);
            a2 = fma(x2, y2, a2);
            a3 = fma(x3, y3, a3);
          }
          for (; i < n; i += g) ga = fma(gp[i], gq[i], ga);
          ga = (ga + a1) + (a2 + a3);
        }
        for (int o = g >> 1; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o, g);
        T cs = 1, sn = 0;
        if (act) act = ga != (T)0 && ga * ga > tol2 * al * be && jacobi_rot(al, be, ga, cs, sn);
        if (act) {
          T *gp = G + ld * p, *gq = G + ld * q, *vp = V + ld * p, *vq = V + ld * q;
          // all loads of a row pair before its stores, two rows at a time: the four columns are
          // distinct, but the compiler cannot prove it, so each store would otherwise wait
          int i = li;
          for (; i + g < n; i += 2 * g) {
            const T x0 = gp[i], y0 = gq[i], x1 = gp[i + g], y1 = gq[i + g];
            const T u0 = vp[i], w0 = vq[i], u1 = vp[i + g], w1 = vq[i + g];
            gp[i] = fma(-sn, y0, cs * x0);
            gq[i] = fma(sn, x0, cs * y0);
            gp[i + g] = fma(-sn, y1, cs * x1);
            gq[i + g] = fma(sn, x1, cs * y1);
            vp[i] = fma(-sn, w0, cs * u0);
            vq[i] = fma(sn, u0, cs * w0);
            vp[i + g] = fma(-sn, w1, cs * u1);
            vq[i + g] = fma(sn, u1, cs * w1);
          }
          for (; i < n; i += g) {
            const T x = gp[i], y = gq[i];
            gp[i] = fma(-sn, y, cs * x);
            gq[i] = fma(sn, x, cs * y);
            const T xv = vp[i], yv = vq[i];
            vp[i] = fma(-sn, yv, cs * xv);
            vq[i] = fma(sn, xv, cs * yv);
          }
          if (li == 0) {
            const T c2 = cs * cs, s2 = sn * sn, cg = (T)2 * cs * sn * ga;
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

// FP32 sweeps for n <= 32 (same ordering, tolerance, zero-column rule and stopping rule as
// jacobi_sweeps_t<float>): one warp per column pair and one lane per row, so a pair's dot product
// is one product per lane and one butterfly sum, every lane forms the rotation parameters itself
// (no broadcast), the tournament positions advance by an add and a compare, and the parameters use
// the approximate FP32 reciprocal and reciprocal square root (cs = 1 / sqrt(1 + t^2), sn = cs t is
// orthogonal to FP32 rounding whatever t's last bits). A round is then a short dependent chain
// (loads, one product, five shuffles, ~12 ALU operations, the stores, the barrier); the generic
// loop costs several times more per round in instruction latency. These sweeps only precondition:
// the FP64 phase that follows fixes the result to FP64 accuracy.
static __device__ __noinline__ int jacobi_sweeps_f32_narrow(float *G, float *V, int n, int ld, float *nrm,
                                                            int max_sweeps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int np = (n + 1) & ~1, P = np / 2, R = np - 1;
  const bool row = lane < n;
  const float eps = FLT_EPSILON;
  const float tolj = 16.0f * eps * sqrtf((float)(n > 4 ? n : 4));
  const float tol2 = tolj * tolj;
  __shared__ float s_fro2;
  __shared__ int s_rot;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = warp; j < n; j += nw) {  // exact column norms at the start of each sweep
      const float x = row ? G[lane + ld * j] : 0.0f;
      float s = x * x;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) nrm[j] = s;
    }
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    if (sweep == 0) {
      if (threadIdx.x == 0) {
        float f = 0.0f;
        for (int j = 0; j < n; ++j) f += nrm[j];
        s_fro2 = f;
      }
      __syncthreads();
    }
    const float floor2 = (float)n * eps * (float)n * eps * s_fro2;
    for (int round = 0; round < R; ++round) {
      for (int pr = warp; pr < P; pr += nw) {  // warp-uniform
        int p, q;
        if (pr == 0) {
          p = round;
          q = np - 1;
        } else {
          p = round + pr;
          p = p >= R ? p - R : p;
          q = round - pr;
          q = q < 0 ? q + R : q;
          if (p > q) {
            const int x = p;
            p = q;
            q = x;
          }
        }
        const bool pair = q < n;  // the extra position of an odd n pairs with nothing
        const float al = pair ? nrm[p] : 0.0f, be = pair ? nrm[q] : 0.0f;
        float *gp = G + ld * p, *gq = G + ld * (pair ? q : p), *vp = V + ld * p, *vq = V + ld * (pair ? q : p);
        const float x = row ? gp[lane] : 0.0f, y = row ? gq[lane] : 0.0f;
        const float u = row ? vp[lane] : 0.0f, w = row ? vq[lane] : 0.0f;
        float ga = x * y;
        for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        bool act = pair && al > floor2 && be > floor2 && ga != 0.0f && ga * ga > tol2 * al * be;
        float cs = 1.0f, sn = 0.0f;
        if (act) {
          const float z = __fdividef(be - al, 2.0f * ga);
          const float zz = fmaf(z, z, 1.0f);
          const float t = copysignf(__fdividef(1.0f, fabsf(z) + zz * rsqrtf(zz)), z);
          act = isfinite(zz) && t != 0.0f && isfinite(t);
          cs = rsqrtf(fmaf(t, t, 1.0f));
          sn = cs * t;
        }
        if (act) {
          if (row) {
            gp[lane] = fmaf(-sn, y, cs * x);
            gq[lane] = fmaf(sn, x, cs * y);
            vp[lane] = fmaf(-sn, w, cs * u);
            vq[lane] = fmaf(sn, u, cs * w);
          }
          if (lane == 0) {
            const float c2 = cs * cs, s2 = sn * sn, cg = 2.0f * cs * sn * ga;
            nrm[p] = fmaf(c2, al, fmaf(s2, be, -cg));
            nrm[q] = fmaf(s2, al, fmaf(c2, be, cg));
            s_rot = 1;
          }
        }
      }
      __syncthreads();
    }
    const int rotated = s_rot;
    __syncthreads();
    if (!rotated) break;
  }
  return sweep + 1;
}

// Doubles of work area jacobi_sweeps_mixed needs for an n x n matrix.
__host__ __device__ inline int64_t jacobi_mixed_work(int64_t n) { return 3 * n * (n + 1); }
// C (n x n, ld ldc) = op(X) op(Y) (+ X when acc) for n x n operands with leading dimensions ldx,
// ldy (tx / ty: transpose), one output per thread per pass, two accumulators. Spread over a
// cluster of nc CTAs (nc = 1: this CTA alone): CTA `me` computes the output columns
// j = me, me + nc, ... and stores each value into every CTA's copy of C (visible after the next
// cluster_sync_all). GB300 issues FP64 at 1/64 of the FP32 rate, so a 32 x 32 x 32 product is
// ~16K cycles of one SM's FP64 pipes whatever the thread count: the cluster divides that by nc.
static __device__ void cta_nn_product(double *C, int ldc, const double *X, int ldx, bool tx, const double *Y,
                                      int ldy, bool ty, int n, bool acc, unsigned nc, unsigned me) {
  const int ncol = (n - (int)me + (int)nc - 1) / (int)nc;
  for (int idx = threadIdx.x; idx < n * ncol; idx += blockDim.x) {
    const int i = idx % n, j = (int)me + (int)nc * (idx / n);
    double s0 = acc ? X[i + ldx * j] : 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < n; l += 2) {
      s0 = fma(tx ? X[l + ldx * i] : X[i + ldx * l], ty ? Y[j + ldy * l] : Y[l + ldy * j], s0);
      s1 = fma(tx ? X[l + 1 + ldx * i] : X[i + ldx * (l + 1)], ty ? Y[j + ldy * (l + 1)] : Y[l + 1 + ldy * j], s1);
    }
    if (l < n) s0 = fma(tx ? X[l + ldx * i] : X[i + ldx * l], ty ? Y[j + ldy * l] : Y[l + ldy * j], s0);
    if (nc == 1)
      C[i + ldc * j] = s0 + s1;
    else
      dsmem_put_all(C + i + ldc * j, s0 + s1, nc);
  }
}

// R = I - X^T X (n x n, ld ldr) for X (ld ldx): the upper triangle computed (entries
// me, me + nc, ... of its packed order on CTA me of nc), the lower mirrored, stored as
// cta_nn_product stores.
static __device__ void cta_gram_residual(double *R, int ldr, const double *X, int ldx, int n, unsigned nc,
                                         unsigned me) {
  const int m = n * (n + 1) / 2;
  for (int idx = (int)me + (int)nc * threadIdx.x; idx < m; idx += (int)nc * blockDim.x) {
    int i, j;
    packed_upper(idx, false, i, j);
    const double *xi = X + ldx * i, *xj = X + ldx * j;
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < n; l += 2) {
      s0 = fma(xi[l], xj[l], s0);
      s1 = fma(xi[l + 1], xj[l + 1], s1);
    }
    if (l < n) s0 = fma(xi[l], xj[l], s0);
    const double r = (i == j ? 1.0 : 0.0) - (s0 + s1);
    if (nc == 1) {
      R[i + ldr * j] = r;
      R[j + ldr * i] = r;
    } else {
      dsmem_put_all(R + i + ldr * j, r, nc);
      if (i != j) dsmem_put_all(R + j + ldr * i, r, nc);
    }
  }
}

// Non-negative doubles order like their bit patterns: maxima of |x| on the integer pipe.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Extra doubles the matrix-product refinement (jacobi_refine) needs after the sweeps' area.
__host__ __device__ inline int64_t jacobi_refine_work(int64_t n) { return 7 * n * (n + 1); }

// Whether the product refinement can succeed, judged from the FP32 sweeps' squared column norms nf
// (the singular values to FP32 accuracy, up to a common scale): all of them above an FP32 noise
// floor (4 sqrt(n) FLT_EPSILON sigma_max) and no two within 1e-3 relative of each other. Declining
// here skips the refinement's O(n^3) products where its own FP64 checks would reject the matrix
// (exactly rank-deficient or clustered spectra); an accepted matrix is still checked there. All
// threads of the CTA call it; the result is uniform.
static __device__ __noinline__ bool jacobi_refine_plausible(const float *nf, int n) {
  __shared__ float s_mx;
  __shared__ int s_ok;
  if (threadIdx.x < 32) {
    float mx = 0.0f;
    for (int i = threadIdx.x; i < n; i += 32) mx = fmaxf(mx, nf[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) {
      s_mx = sqrtf(mx);
      s_ok = mx > 0.0f && isfinite(mx) ? 1 : 0;
    }
  }
  __syncthreads();
  const float floor_ = 4.0f * sqrtf((float)n) * FLT_EPSILON * s_mx;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float si = sqrtf(fmaxf(nf[i], 0.0f));
    bad |= !(si > floor_);
    for (int j = 0; j < i; ++j) {
      const float sj = sqrtf(fmaxf(nf[j], 0.0f));
      bad |= fabsf(si - sj) <= 1e-3f * fmaxf(si, sj);
    }
  }
  if (bad) s_ok = 0;  // benign race: every writer stores 0
  __syncthreads();
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

// Matrix-product refinement of an SVD (Ogita and Aishima, "Iterative refinement for singular value
// decomposition based on matrix multiplication", 2020), restated. A (n x n, ld n) is the matrix,
// Vin (ld ldv) approximate right singular vectors (the FP32 sweeps' result, widened). With
// U = A V diag(1/sigma), a step forms R = I - U^T U, S = I - V^T V and T = U^T A V, and the
// first-order corrections F, Gc with U <- U (I + F), V <- V (I + Gc) such that both stay
// orthonormal and U^T A V becomes diagonal: sigma_i = t_ii / (1 - (r_ii + s_ii) / 2),
// f_ii = r_ii / 2, g_ii = s_ii / 2, and for i < j, with a = -t_ij - sigma_j r_ij and
// b = -t_ji - sigma_j s_ij, f_ij = (-sigma_j a - sigma_i b) / (sigma_j^2 - sigma_i^2),
// g_ij = (-sigma_i a - sigma_j b) / (sigma_j^2 - sigma_i^2), f_ji = r_ij - f_ij, g_ji = s_ij - g_ij.
// The error contracts quadratically while the singular values are separated: from the FP32 sweeps'
// result two steps reach FP64 accuracy, with products only (no sequential rotation rounds). A step
// whose residual e = max(|R|, |S|, |offdiag T| / sigma_max) is at most 1e-9 is the last (the error
// after it is ~e^2, below FP64 rounding); at most three steps run. On success A becomes
// U diag(sigma) (columns sigma_j u_j, the one-sided Jacobi convention), Vout (ld n) the refined V,
// and the function returns true. It returns false, leaving A and Vin untouched, when two singular
// values lie within 1e-3 relative of each other, one is below n eps sigma_max, the first residual
// exceeds 1e-2, or the third is still above 1e-9; the caller then runs the FP64 sweeps.
// wk: jacobi_refine_work(n) doubles. All threads of the CTA call it. With `cluster`, every CTA of
// the thread-block cluster calls it with identical A and Vin in its own shared memory (wk too):
// the products and the corrections are split over the CTAs and every result is stored into each
// CTA's copy, one cluster barrier per phase; the checks run on identical data in every CTA, so all
// take the same branches, and every CTA ends with the same A and Vout.
static __device__ __noinline__ bool jacobi_refine(double *A, const double *Vin, int ldv, double *Vout, int n,
                                                  double *wk, bool cluster = false) {
  const int ld = n + 1, nthr = blockDim.x;
  const unsigned nc = cluster ? cluster_nctarank() : 1u, me = cluster ? cluster_ctarank() : 0u;
  double *U = wk, *V = U + n * ld, *H = V + n * ld, *R = H + n * ld, *Sm = R + n * ld, *Tm = Sm + n * ld;
  double *Fm = Tm + n * ld;  // F; Gc goes into H (A V is recomputed each step)
  __shared__ double s_sig[1024];
  __shared__ float s_sigf[1024];
  __shared__ unsigned long long s_rs, s_t;
  __shared__ double s_e;
  __shared__ int s_bad;
  auto sync_all = [nc]() {
    if (nc > 1)
      cluster_sync_all();
    else
      __syncthreads();
  };
  for (int idx = threadIdx.x; idx < n * n; idx += nthr) {
    const int i = idx % n, j = idx / n;
    V[i + ld * j] = Vin[i + ldv * j];
  }
  __syncthreads();
  cta_nn_product(H, ld, A, n, false, V, ld, false, n, false, nc, me);  // H = A V
  sync_all();
  for (int j = threadIdx.x; j < n; j += nthr) {  // one reciprocal per column
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < n; i += 2) {
      s0 = fma(H[i + ld * j], H[i + ld * j], s0);
      s1 = fma(H[i + 1 + ld * j], H[i + 1 + ld * j], s1);
    }
    if (i < n) s0 = fma(H[i + ld * j], H[i + ld * j], s0);
    const double sj = sqrt(s0 + s1);
    s_sig[j] = sj > 0.0 ? 1.0 / sj : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += nthr) {
    const int i = idx % n, j = idx / n;
    U[i + ld * j] = H[i + ld * j] * s_sig[j];
  }
  __syncthreads();
  bool done = false;
  for (int step = 0; step < 3 && !done; ++step) {
    cta_gram_residual(R, ld, U, ld, n, nc, me);   // R = I - U^T U
    cta_gram_residual(Sm, ld, V, ld, n, nc, me);  // S = I - V^T V
    if (step > 0) cta_nn_product(H, ld, A, n, false, V, ld, false, n, false, nc, me);
    if (threadIdx.x == 0) {
      s_rs = 0ull;
      s_t = 0ull;
      s_bad = 0;
    }
    sync_all();
    cta_nn_product(Tm, ld, U, ld, true, H, ld, false, n, false, nc, me);  // T = U^T A V
    sync_all();
    for (int i = threadIdx.x; i < n; i += nthr) {
      const double s = Tm[i + ld * i] / (1.0 - 0.5 * (R[i + ld * i] + Sm[i + ld * i]));
      s_sig[i] = s;
      s_sigf[i] = (float)fabs(s);
    }
    // residual maxima as bit patterns (integer pipe); off-diagonal T scaled by sigma_max once
    {
      unsigned long long mrs = 0ull, mt = 0ull;
      for (int idx = threadIdx.x; idx < n * n; idx += nthr) {
        const int i = idx % n, j = idx / n;
        const unsigned long long a = abs_bits(R[i + ld * j]), b = abs_bits(Sm[i + ld * j]);
        mrs = a > mrs ? a : mrs;
        mrs = b > mrs ? b : mrs;
        const unsigned long long t = i != j ? abs_bits(Tm[i + ld * j]) : 0ull;
        mt = t > mt ? t : mt;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, mrs, o), y = __shfl_xor_sync(0xffffffffu, mt, o);
        mrs = x > mrs ? x : mrs;
        mt = y > mt ? y : mt;
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMax(&s_rs, mrs);
        atomicMax(&s_t, mt);
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // sigma_max, then the checks in FP32 (separation at 1e-3 needs no more)
      float mx = 0.0f;
      for (int i = threadIdx.x; i < n; i += 32) mx = fmaxf(mx, s_sigf[i]);
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      double smx = 0.0;
      for (int i = threadIdx.x; i < n; i += 32) smx = s_sigf[i] == mx ? fabs(s_sig[i]) : smx;
      for (int o = 16; o > 0; o >>= 1) smx = fmax(smx, __shfl_xor_sync(0xffffffffu, smx, o));
      bool bad = !(mx > 0.0f) || !isfinite(mx);
      const float floor_ = (float)n * FLT_EPSILON * mx;  // a bound below sigma_i <= n eps sigma_max
      for (int i = threadIdx.x; i < n; i += 32) {
        const float si = s_sigf[i];
        bad |= !(si > floor_) || !(s_sig[i] > (double)n * DBL_EPSILON * smx);
        for (int j = 0; j < i; ++j) bad |= fabsf(si - s_sigf[j]) <= 1e-3f * fmaxf(si, s_sigf[j]);
      }
      bad = __any_sync(0xffffffffu, bad);
      if (threadIdx.x == 0) {
        const double e = fmax(__longlong_as_double((long long)s_rs), __longlong_as_double((long long)s_t) / smx);
        bad |= !(e <= 1e-2) || (step == 2 && !(e <= 1e-9));
        s_bad = bad ? 1 : 0;
        s_e = e;
      }
    }
    __syncthreads();
    if (s_bad) return false;
    done = s_e <= 1e-9;
    // corrections, one FP64 division per pair: F into Fm, Gc into H
    for (int i = (int)me + (int)nc * threadIdx.x; i < n; i += (int)nc * nthr) {
      const double f = 0.5 * R[i + ld * i], g = 0.5 * Sm[i + ld * i];
      if (nc == 1) {
        Fm[i + ld * i] = f;
        H[i + ld * i] = g;
      } else {
        dsmem_put_all(Fm + i + ld * i, f, nc);
        dsmem_put_all(H + i + ld * i, g, nc);
      }
    }
    const int npair = n * (n - 1) / 2;
    for (int idx = (int)me + (int)nc * threadIdx.x; idx < npair; idx += (int)nc * nthr) {
      int a, b;
      packed_upper(idx, true, a, b);  // a < b
      const double sa = s_sig[a], sb = s_sig[b], rab = R[a + ld * b], sab = Sm[a + ld * b];
      const double aa = -Tm[a + ld * b] - sb * rab;
      const double bb = -Tm[b + ld * a] - sb * sab;
      const double inv = 1.0 / ((sb - sa) * (sb + sa));
      const double fab = (-sb * aa - sa * bb) * inv, gab = (-sa * aa - sb * bb) * inv;
      if (nc == 1) {
        Fm[a + ld * b] = fab;
        H[a + ld * b] = gab;
        Fm[b + ld * a] = rab - fab;
        H[b + ld * a] = sab - gab;
      } else {
        dsmem_put_all(Fm + a + ld * b, fab, nc);
        dsmem_put_all(H + a + ld * b, gab, nc);
        dsmem_put_all(Fm + b + ld * a, rab - fab, nc);
        dsmem_put_all(H + b + ld * a, sab - gab, nc);
      }
    }
    sync_all();
    // U <- U + U F into R's area, V <- V + V Gc into S's area, then the areas swap
    cta_nn_product(R, ld, U, ld, false, Fm, ld, false, n, true, nc, me);
    cta_nn_product(Sm, ld, V, ld, false, H, ld, false, n, true, nc, me);
    sync_all();
    double *x = U;
    U = R;
    R = x;
    x = V;
    V = Sm;
    Sm = x;
  }
  if (!done) return false;
  // sigma from the last step's diagonal formula; A <- U diag(sigma), Vout <- V
  for (int idx = threadIdx.x; idx < n * n; idx += nthr) {
    const int i = idx % n, j = idx / n;
    A[i + n * j] = U[i + ld * j] * s_sig[j];
    Vout[i + n * j] = V[i + ld * j];
  }
  __syncthreads();
  return true;
}

// Mixed-precision one-sided Jacobi (the preconditioned scheme of Gao, Ma and Shao, "A mixed
// precision Jacobi SVD algorithm", 2022): the sweeps run to convergence in FP32 on a copy of G
// (scaled by a power of two into FP32 range), the FP32 right vectors V0 are made orthonormal to
// FP64 rounding by two Newton-Schulz steps V <- V (3 I - V^T V) / 2 (quadratic: ~1e-6 -> 1e-12 ->
// rounding level), and the FP64 sweeps then run on G V0 with V accumulated from V0. The columns
// of G V0 are orthogonal to FP32 accuracy, so the FP64 phase converges in two or three sweeps
// (the last one only confirms) instead of six to eight: most of the O(n^3) work per sweep moves to
// the FP32 pipe, 64 times wider than FP64 on GB300. Results: G V = U S with V orthogonal to FP64
// rounding, as plain FP64 sweeps give. V on entry is ignored (the identity is assumed).
// work: jacobi_mixed_work(n) doubles. Returns the number of FP64 sweeps. The two phases are
// separate functions so that a cluster kernel can run the first on one CTA and share its result.
//
// FP32 phase: leaves the widened FP32 right vectors V0 in work + n (n + 1) (ld n + 1); G is read.
static __device__ __noinline__ void jacobi_fp32_phase(const double *G, int n, double *nrm, double *work) {
  const int nthr = blockDim.x;
  const int nn = n * n;
  // padded working copies (leading dimension n + 1): columns i and i + 1 start in different
  // shared-memory banks, so neither the pairs a warp rotates together nor a column-per-lane
  // product serialise on one bank. work: Gp, Vp, Tp (n x (n + 1) doubles each); the FP32 copies
  // live in Tp during the FP32 phase, their norms in nrm.
  const int ld = n + 1, np = n * ld;
  double *Vp = work + np, *Tp = work + 2 * np;
  float *Gf = reinterpret_cast<float *>(Tp), *Vf = Gf + np, *nf = reinterpret_cast<float *>(nrm);
  __shared__ double s_scale;
  // power-of-two scale bringing ||G||_F near 1 (FP32 range; exact in both directions)
  for (int j = threadIdx.x; j < n; j += nthr) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(G[i + n * j], G[i + n * j], s);
    nrm[j] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int j = 0; j < n; ++j) f += nrm[j];
    const int e = f > 0.0 && isfinite(f) ? (((int)((__double_as_longlong(f) >> 52) & 0x7FF) - 1023) >> 1) : 0;
    s_scale = pow2(-e);
  }
  __syncthreads();
  const double sc = s_scale;
  for (int idx = threadIdx.x; idx < nn; idx += nthr) {
    const int i = idx % n, j = idx / n;
    Gf[i + ld * j] = (float)(G[idx] * sc);
    Vf[i + ld * j] = i == j ? 1.0f : 0.0f;
  }
  __syncthreads();
  if (n <= 32)
    jacobi_sweeps_f32_narrow(Gf, Vf, n, ld, nf, 40);
  else
    jacobi_sweeps_t<float>(Gf, Vf, n, ld, nf, 40);
  for (int idx = threadIdx.x; idx < nn; idx += nthr) {
    const int i = idx % n, j = idx / n;
    Vp[i + ld * j] = (double)Vf[i + ld * j];
  }
  __syncthreads();
}

// FP64 phase from V0 (jacobi_fp32_phase's result in work): G V = U S with V orthogonal to FP64
// rounding. G (ld n) and V (ld n) are overwritten. Returns the number of FP64 sweeps.
static __device__ __noinline__ int jacobi_fp64_finish(double *G, double *V, int n, double *nrm, double *work) {
  const int nthr = blockDim.x;
  const int nn = n * n;
  const int ld = n + 1, np = n * ld;
  double *Gp = work, *Vp = work + np, *Tp = work + 2 * np;
  // Newton-Schulz steps: T1 = V^T V (in Gp), V <- 1.5 V - 0.5 V T1 (into Tp; the FP32 copies
  // are dead now), then the roles of Vp and Tp swap. Lane i reads row l of column i of V (stride
  // n + 1: conflict-free) or row i of column l; the other operand is a broadcast.
  for (int it = 0; it < 2; ++it) {
    for (int idx = threadIdx.x; idx < nn; idx += nthr) {
      const int i = idx % n, j = idx / n;
      const double *vi = Vp + ld * i, *vj = Vp + ld * j;
      double s0 = 0.0, s1 = 0.0;
      int l = 0;
      for (; l + 1 < n; l += 2) {
        s0 = fma(vi[l], vj[l], s0);
        s1 = fma(vi[l + 1], vj[l + 1], s1);
      }
      if (l < n) s0 = fma(vi[l], vj[l], s0);
      Gp[i + ld * j] = s0 + s1;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nn; idx += nthr) {
      const int i = idx % n, j = idx / n;
      const double *t = Gp + ld * j;
      double s0 = 0.0, s1 = 0.0;
      int l = 0;
      for (; l + 1 < n; l += 2) {
        s0 = fma(Vp[i + ld * l], t[l], s0);
        s1 = fma(Vp[i + ld * (l + 1)], t[l + 1], s1);
      }
      if (l < n) s0 = fma(Vp[i + ld * l], t[l], s0);
      Tp[i + ld * j] = fma(-0.5, s0 + s1, 1.5 * Vp[i + ld * j]);
    }
    __syncthreads();
    double *x = Vp;
    Vp = Tp;
    Tp = x;
  }
  // Gp <- G V0
  for (int idx = threadIdx.x; idx < nn; idx += nthr) {
    const int i = idx % n, j = idx / n;
    const double *v = Vp + ld * j;
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < n; l += 2) {
      s0 = fma(G[i + n * l], v[l], s0);
      s1 = fma(G[i + n * (l + 1)], v[l + 1], s1);
    }
    if (l < n) s0 = fma(G[i + n * l], v[l], s0);
    Gp[i + ld * j] = s0 + s1;
  }
  __syncthreads();
  const int sweeps = jacobi_sweeps_t<double>(Gp, Vp, n, ld, nrm, 60);
  for (int idx = threadIdx.x; idx < nn; idx += nthr) {
    const int i = idx % n, j = idx / n;
    G[idx] = Gp[i + ld * j];
    V[idx] = Vp[i + ld * j];
  }
  __syncthreads();
  return sweeps;
}

// Both phases; with refine_work (jacobi_refine_work(n) doubles) the FP64 phase is replaced by the
// product refinement whenever that accepts (separated singular values; it then returns 0).
static __device__ __noinline__ int jacobi_sweeps_mixed(double *G, double *V, int n, double *nrm, double *work,
                                                       double *refine_work = nullptr) {
  jacobi_fp32_phase(G, n, nrm, work);
  if (refine_work && n <= 1024 && jacobi_refine_plausible(reinterpret_cast<const float *>(nrm), n) &&
      jacobi_refine(G, work + n * (n + 1), n + 1, V, n, refine_work))
    return 0;
  return jacobi_fp64_finish(G, V, n, nrm, work);
}

}  // namespace tnr
