// Device helpers shared by several translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace tnr {

__device__ __forceinline__ double dwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Position (i, j), i <= j (strict: i < j), of entry idx of the packed upper triangle of an n x n
// matrix, column by column. The FP32 square root is corrected by integer steps.
__device__ __forceinline__ void packed_upper(int idx, bool strict, int &i, int &j) {
  const int s = strict ? 1 : 0;  // strict: column j holds j entries, else j + 1
  int c = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f) + s;
  auto start = [s](int col) { return s ? col * (col - 1) / 2 : col * (col + 1) / 2; };
  while (c > 0 && start(c) > idx) --c;
  while (start(c + 1) <= idx) ++c;
  j = c;
  i = idx - start(c);
}

// Jacobi rotation (c, s) annihilating gamma = g_p^T g_q for alpha = ||g_p||^2, beta = ||g_q||^2:
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (beta - alpha) / (2 gamma). The angle
// only steers convergence, so t is formed in FP32 after an exact power-of-two scaling; c =
// 1 / sqrt(1 + t^2) is refined to FP64 by two Newton steps from the FP32 estimate, so c^2 + s^2
// = 1 to FP64 rounding. No FP64 division or square root (long sequences on GB300's FP64 pipe).
// Returns false when the rotation is negligible.
__device__ __forceinline__ bool jacobi_rotation(double al, double be, double ga, double &cs, double &sn) {
  // exact power-of-two scale 2^-e with e the binary exponent of 2*gamma (bit manipulation,
  // no library calls): 2*gamma*scale lies in [1, 2)
  const long long eb = (__double_as_longlong(2.0 * ga) >> 52) & 0x7FF;
  if (eb == 0 || eb == 0x7FF) return false;  // gamma subnormal or non-finite: negligible/invalid
  const double scale = __longlong_as_double((2046LL - eb) << 52);
  const double diff = (be - al) * scale, den = (2.0 * ga) * scale;
  const float zf = (float)diff / (float)den;
  if (!isfinite(zf)) return false;
  const float tf = copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
  if (tf == 0.0f) return false;
  const double t = (double)tf;
  const double x = fma(t, t, 1.0);
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  cs = y;
  sn = y * t;
  return true;
}

// Householder reflector parameters (LAPACK dlarfg convention) for x = (alpha, x_2..) with
// sig = ||x_2..||^2 > 0: beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta = 1 + |alpha| r
// and scal = 1 / (alpha - beta) = sign(alpha) r / tau with r = 1 / ||x|| (v = x_2.. * scal,
// v_1 = 1). Written without FP64 division or square root, with a short dependent chain (these
// parameters sit on the critical path of every pivot step): r from an FP32 estimate refined by
// one third-order step r (1 + e/2 + 3e^2/8), e = 1 - n r^2 (the Taylor series of (1 - e)^(-1/2)),
// and 1 / tau (tau in [1, 2], no range reduction) from an FP32 reciprocal refined by
// q (1 + e + e^2), e = 1 - tau q (the geometric series). The FP32 estimates' relative error
// (< 2^-21) leaves O(2^-63) after the step, below FP64 rounding.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

__device__ __forceinline__ void householder_params(double alpha, double sig, double &beta, double &tau,
                                                   double &scal) {
  const double n2 = fma(alpha, alpha, sig);
  // exact power-of-two range reduction so the FP32 seed never overflows or underflows
  const int k = ((int)((__double_as_longlong(n2) >> 52) & 0x7FF) - 1023) >> 1;  // floor(e / 2)
  const double n2s = n2 * pow2(-2 * k);                                            // in [1, 4)
  double r = (double)rsqrtf((float)n2s);
  const double e = fma(-n2s * r, r, 1.0);
  r = fma(r * e, fma(0.375, e, 0.5), r);
  r *= pow2(-k);  // 1 / ||x||
  const double sgn = alpha < 0.0 ? -1.0 : 1.0;
  beta = -sgn * (n2 * r);
  tau = fma(fabs(alpha), r, 1.0);
  double q = (double)(1.0f / (float)tau);
  const double et = fma(-tau, q, 1.0);
  q = fma(q, fma(et, et, et), q);
  scal = (sgn * r) * q;
}

// 1 / sqrt(x) for finite x > 0 to FP64 accuracy without the FP64 square-root / division
// sequences: exact power-of-two range reduction, FP32 seed, two Newton steps (24 -> 48 -> 53 bits).
__device__ __forceinline__ double rsqrt_f64(double x) {
  const int k = ((int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023) >> 1;  // floor(e / 2)
  const double xs = x * pow2(-2 * k);                                          // in [1, 4)
  double r = (double)rsqrtf((float)xs);
  r = r * fma(-0.5 * xs, r * r, 1.5);
  r = r * fma(-0.5 * xs, r * r, 1.5);
  return r * pow2(-k);
}

// SplitMix64 (Steele, Lea, Flood 2014) at counter n of the stream with the given seed.
static __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}


// Normal draw m of the Lemma 5.1 random MPO: uniforms ((z >> 11) + 1) 2^-53 in (0, 1] from
// counters 2m and 2m+1, Box-Muller cosine branch.
static __device__ __forceinline__ double omega_normal(uint64_t seed, uint64_t m) {
  const double u1 = (double)((splitmix64_at(seed, 2 * m) >> 11) + 1) * 0x1.0p-53;
  const double u2 = (double)((splitmix64_at(seed, 2 * m + 1) >> 11) + 1) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos((2.0 * M_PI) * u2);
}

// 1 / x for finite x > 0: exact power-of-two range reduction, FP32 reciprocal seed, two Newton steps.
__device__ __forceinline__ double rcp_f64(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
  const double xs = x * pow2(-e);  // in [1, 2)
  double q = (double)(1.0f / (float)xs);
  q = q * fma(-xs, q, 2.0);
  q = q * fma(-xs, q, 2.0);
  return q * pow2(-e);
}

}  // namespace tnr
