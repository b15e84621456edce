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
// The sweeps are written once for FP32 and FP64; jacobi_sweeps_mixed runs them in FP32 first and
// finishes in FP64 (see there), which is what the SVD kernels call.
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

// Doubles of work area jacobi_sweeps_mixed needs for an n x n matrix.
__host__ __device__ inline int64_t jacobi_mixed_work(int64_t n) { return 3 * n * (n + 1); }
// Extra doubles the matrix-product refinement (jacobi_refine) needs after that area.
__host__ __device__ inline int64_t jacobi_refine_work(int64_t n) { return 7 * n * (n + 1); }

// C (n x n, ld ldc) = op(X) op(Y) for n x n operands with leading dimensions ldx, ldy
// (tx / ty: transpose), by the whole CTA, one output per thread per pass, two accumulators.
static __device__ void cta_nn_product(double *C, int ldc, const double *X, int ldx, bool tx, const double *Y,
                                      int ldy, bool ty, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, j = idx / n;
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < n; l += 2) {
      s0 = fma(tx ? X[l + ldx * i] : X[i + ldx * l], ty ? Y[j + ldy * l] : Y[l + ldy * j], s0);
      s1 = fma(tx ? X[l + 1 + ldx * i] : X[i + ldx * (l + 1)], ty ? Y[j + ldy * (l + 1)] : Y[l + 1 + ldy * j], s1);
    }
    if (l < n) s0 = fma(tx ? X[l + ldx * i] : X[i + ldx * l], ty ? Y[j + ldy * l] : Y[l + ldy * j], s0);
    C[i + ldc * j] = s0 + s1;
  }
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
// The error contracts quadratically while the singular values are separated: two steps take the
// FP32 result to FP64 accuracy, with products only (no sequential rotation rounds). On success A
// becomes U diag(sigma) (columns sigma_j u_j, the one-sided Jacobi convention), Vout (ld n) the refined V,
// and the function returns true. It returns false, leaving A and Vin untouched, when two singular
// values lie within 1e-3 relative of each other, one is below n eps sigma_max, or the residual has
// not dropped below 1e-9 after the first step; the caller then runs the FP64 sweeps.
// wk: jacobi_refine_work(n) doubles.
static __device__ __noinline__ bool jacobi_refine(double *A, const double *Vin, int ldv, double *Vout, int n,
                                                  double *wk) {
  const int ld = n + 1;
  double *U = wk, *V = U + n * ld, *H = V + n * ld, *R = H + n * ld, *Sm = R + n * ld, *Tm = Sm + n * ld;
  double *Fm = Tm + n * ld;  // F, then Gc written over R / S as they are consumed
  __shared__ double s_sig[1024];
  __shared__ int s_ok;
  __shared__ double s_err;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, j = idx / n;
    V[i + ld * j] = Vin[i + ldv * j];
  }
  __syncthreads();
  cta_nn_product(H, ld, A, n, false, V, ld, false, n);  // H = A V
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s0 = 0.0;
    for (int i = 0; i < n; ++i) s0 = fma(H[i + ld * j], H[i + ld * j], s0);
    s_sig[j] = sqrt(s0);
  }
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, j = idx / n;
    U[i + ld * j] = s_sig[j] > 0.0 ? H[i + ld * j] / s_sig[j] : 0.0;
  }
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    cta_nn_product(R, ld, U, ld, true, U, ld, false, n);   // U^T U
    cta_nn_product(Sm, ld, V, ld, true, V, ld, false, n);  // V^T V
    if (step > 0) cta_nn_product(H, ld, A, n, false, V, ld, false, n);
    __syncthreads();
    cta_nn_product(Tm, ld, U, ld, true, H, ld, false, n);  // T = U^T A V
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {  // R = I - U^T U, S = I - V^T V
      const int i = idx % n, j = idx / n;
      R[i + ld * j] = (i == j ? 1.0 : 0.0) - R[i + ld * j];
      Sm[i + ld * j] = (i == j ? 1.0 : 0.0) - Sm[i + ld * j];
    }
    __syncthreads();
    // sigma from the diagonal (one thread per value), then the checks spread over the CTA (FP64
    // work on one thread would hold its pipe ~64 cycles per instruction)
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      s_sig[i] = Tm[i + ld * i] / (1.0 - 0.5 * (R[i + ld * i] + Sm[i + ld * i]));
    if (threadIdx.x == 0) s_err = 0.0;
    __syncthreads();
    double smax = 0.0;
    for (int i = 0; i < n; ++i) smax = fmax(smax, fabs(s_sig[i]));
    {
      bool bad = false;
      double err = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bad |= !(s_sig[i] > (double)n * DBL_EPSILON * smax);
        for (int j = 0; j < i; ++j) bad |= fabs(s_sig[i] - s_sig[j]) <= 1e-3 * fmax(s_sig[i], s_sig[j]);
      }
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        err = fmax(err, fmax(fabs(R[i + ld * j]), fabs(Sm[i + ld * j])));
        if (i != j) err = fmax(err, fabs(Tm[i + ld * j]) / smax);
      }
      for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
      if (bad) s_ok = 0;
      if ((threadIdx.x & 31) == 0 && err > 0.0)  // non-negative doubles order like their bits
        atomicMax(reinterpret_cast<unsigned long long *>(&s_err), (unsigned long long)__double_as_longlong(err));
    }
    __syncthreads();
    if (step == 1 && !(s_err <= 1e-9)) s_ok = 0;
    __syncthreads();
    if (!s_ok) return false;
    // corrections: F into Fm, Gc into H (H = A V is recomputed next step)
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx % n, j = idx / n;
      double f, g;
      if (i == j) {
        f = 0.5 * R[i + ld * i];
        g = 0.5 * Sm[i + ld * i];
      } else {
        const int a_ = i < j ? i : j, b_ = i < j ? j : i;  // solve for the pair (a_, b_), a_ < b_
        const double sa = s_sig[a_], sb = s_sig[b_];
        const double aa = -Tm[a_ + ld * b_] - sb * R[a_ + ld * b_];
        const double bb = -Tm[b_ + ld * a_] - sb * Sm[a_ + ld * b_];
        const double det = sb * sb - sa * sa;
        const double fab = (-sb * aa - sa * bb) / det, gab = (-sa * aa - sb * bb) / det;
        if (i < j) {
          f = fab;
          g = gab;
        } else {
          f = R[a_ + ld * b_] - fab;
          g = Sm[a_ + ld * b_] - gab;
        }
      }
      Fm[i + ld * j] = f;
      H[i + ld * j] = g;
    }
    __syncthreads();
    // U <- U + U F, V <- V + V Gc (products into R / S, then added)
    cta_nn_product(R, ld, U, ld, false, Fm, ld, false, n);
    cta_nn_product(Sm, ld, V, ld, false, H, ld, false, n);
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx % n, j = idx / n;
      U[i + ld * j] += R[i + ld * j];
      V[i + ld * j] += Sm[i + ld * j];
    }
    __syncthreads();
  }
  // sigma from the last step's diagonal formula; A <- U diag(sigma), Vout <- V
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
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
// work: jacobi_mixed_work(n) doubles. Returns the number of FP64 sweeps.
static __device__ __noinline__ int jacobi_sweeps_mixed(double *G, double *V, int n, double *nrm, double *work,
                                                       double *refine_work = nullptr) {
  const int nthr = blockDim.x;
  const int nn = n * n;
  // padded working copies (leading dimension n + 1): columns i and i + 1 start in different
  // shared-memory banks, so neither the pairs a warp rotates together nor a column-per-lane
  // product serialise on one bank. work: Gp, Vp, Tp (n x (n + 1) doubles each); the FP32 copies
  // live in Tp during the FP32 phase, their norms in nrm.
  const int ld = n + 1, np = n * ld;
  double *Gp = work, *Vp = work + np, *Tp = work + 2 * np;
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
  jacobi_sweeps_t<float>(Gf, Vf, n, ld, nf, 40);
  for (int idx = threadIdx.x; idx < nn; idx += nthr) {
    const int i = idx % n, j = idx / n;
    Vp[i + ld * j] = (double)Vf[i + ld * j];
  }
  __syncthreads();
  // separated singular values: finish with the product refinement instead of the FP64 sweeps
  if (refine_work && n <= 1024 && jacobi_refine(G, Vp, ld, V, n, refine_work)) return 0;
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

}  // namespace tnr
