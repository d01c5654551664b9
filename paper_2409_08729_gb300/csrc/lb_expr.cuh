// lb_expr.cuh -- per-pair expressions of the log-Bessel algorithm (device code).
//
// Each function evaluates one of the paper's expressions for one (v, x) pair
// in double precision:
//   mu_K  : large-argument expansion (paper Sec. 3.1 Eq. "log Iv mu k",
//           Sec. 3.2 Eq. "log Kv mu k")
//   U_K   : uniform large-order expansion (Eqs. "log Iv u k", "log Kv u k")
//   series: power series of I_v summed in log scale (Eqs. "Iv infinite series",
//           "ak recurrence", "log Iv")
// The K integral (Eq. "log Kv integral") is warp-cooperative and lives in
// lb_kint.cuh.
#pragma once

#include <math.h>
#include <stdint.h>

template <typename T> __host__ __device__ __forceinline__ T lb_fma(T a, T b, T c);
template <> __host__ __device__ __forceinline__ double lb_fma<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __host__ __device__ __forceinline__ float lb_fma<float>(float a, float b, float c) { return fmaf(a, b, c); }

#include "lb_df.cuh"
#include "debye_uk.h"
#include "lb_fastmath.cuh"
#include "lb_intmath.cuh"

namespace lb {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kHalfLogPi = 0.5723649429247000870717136756012478;   // log(pi)/2
constexpr double kHalfLog2Pi = 0.9189385332046727417803297364056177;  // log(2 pi)/2
constexpr double kHalfLogHalfPi = 0.2257913526447274323630976149;     // log(pi/2)/2

enum Kind { KIND_I = 0, KIND_K = 1 };
enum Region { R_MU20 = 0, R_U13 = 1, R_FALLBACK = 2, R_SPECIAL = 3, R_MU3 = 4, R_U4 = 5, R_U6 = 6, R_U9 = 7 };
enum Mode { MODE_TIGHT = 0, MODE_PAPER_GPU = 1, MODE_PAPER_CPU = 2 };

// ---------------------------------------------------------------------------
// Domain edges (shared convention of the library): returns true and sets *r
// when (v, x) is an edge case; K callers pass |v|.
// ---------------------------------------------------------------------------
// The tests use the IEEE bit patterns (integer instructions): on GB300 a
// double-precision compare costs as much FP64-pipe time as an FMA.
__device__ __forceinline__ bool bits_nan(long long b) { return (b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL; }
__device__ __forceinline__ bool bits_inf(long long b) { return (b & 0x7fffffffffffffffLL) == 0x7ff0000000000000LL; }
__device__ __forceinline__ bool bits_zero(long long b) { return (b & 0x7fffffffffffffffLL) == 0; }
__device__ __forceinline__ bool bits_neg(long long b) { return b < 0 && !bits_zero(b); }

template <int KIND>
__device__ __forceinline__ bool special_value(double v, double x, double* r) {
  const long long bv = __double_as_longlong(v), bx = __double_as_longlong(x);
  if ((bv & 0x7ff0000000000000LL) != 0x7ff0000000000000LL && (bx & 0x7ff0000000000000LL) != 0x7ff0000000000000LL &&
      !bits_neg(bx) && !bits_zero(bx) && (KIND == KIND_K || !bits_neg(bv)))
    return false;                                   // the common case: finite, x > 0, v >= 0 for I
  if (KIND == KIND_I) {
    if (bits_nan(bv) || bits_nan(bx) || bits_neg(bv) || bits_neg(bx) || (bits_inf(bv) && bits_inf(bx))) { *r = __longlong_as_double(0x7ff8000000000000LL); return true; }
    if (bits_inf(bx)) { *r = INFINITY; return true; }
    if (bits_inf(bv)) { *r = -INFINITY; return true; }
    if (bits_zero(bx)) { *r = bits_zero(bv) ? 0.0 : -INFINITY; return true; }
  } else {
    if (bits_nan(bv) || bits_nan(bx) || bits_neg(bx) || (bits_inf(bv) && bits_inf(bx))) { *r = __longlong_as_double(0x7ff8000000000000LL); return true; }
    if (bits_inf(bx)) { *r = -INFINITY; return true; }
    if (bits_zero(bx) || bits_inf(bv)) { *r = INFINITY; return true; }
  }
  return false;
}

// Domain edges of the x-derivatives: d/dx log I_v at x = 0 is 0 for v = 0
// (I_0 = 1 + x^2/4 + ...) and +inf otherwise (I_v ~ (x/2)^v / Gamma(v+1));
// d/dx log K_v at x = 0 is -inf; at x = +inf the derivatives tend to +1 (I)
// and -1 (K); an infinite order gives NaN.
template <int KIND>
__device__ __forceinline__ bool special_dx(double v, double x, double* r) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  if (isnan(v) || isnan(x) || x < 0.0 || isinf(v)) { *r = qnan; return true; }
  if (KIND == KIND_I && v < 0.0) { *r = qnan; return true; }
  if (isinf(x)) { *r = (KIND == KIND_I) ? 1.0 : -1.0; return true; }
  if (x == 0.0) { *r = (KIND == KIND_I) ? (v == 0.0 ? 0.0 : INFINITY) : -INFINITY; return true; }
  return false;
}

// ---------------------------------------------------------------------------
// Region predicates (paper Table "input ranges", Algorithm 1).
// ---------------------------------------------------------------------------
// Paper thresholds as printed.  Comparisons are strict, so a pair exactly on
// a threshold falls through to the next branch.
__device__ __forceinline__ bool paper_mu3(double v, double x) {
  return (x > 1400.0 && v < 3.05) || ((0.6229 * log(x) - 3.2318 > log(v)) && v > 3.1);
}
__device__ __forceinline__ bool paper_mu20(double v, double x) {
  return (x > 30.0 && v < 15.3919) || ((0.5113 * log(x) + 0.7939 > log(v)) && x > 59.6925);
}
__device__ __forceinline__ bool paper_u4(double v, double x) { return (x > 274.2377 && v > 0.3) || v > 163.6993; }
__device__ __forceinline__ bool paper_u6(double v, double x) { return (x > 84.4153 && v > 0.46) || v > 56.9971; }
__device__ __forceinline__ bool paper_u9(double v, double x) { return (x > 35.9074 && v > 0.6) || v > 20.1534; }
__device__ __forceinline__ bool paper_u13(double v, double x) { return (x > 19.6931 && v > 0.7) || v > 12.6964; }

// Tight thresholds: the same two expressions, with the regions shrunk until
// the truncation error of mu_20 and U_13 (measured against an
// extended-precision reference on both sides of every boundary) is below
// 3e-16 of the error scale.  The curved mu_20 boundary
// 0.5113 log x + 0.7939 > log v is replaced by v^2 < 3.24 x, which follows
// the actual validity limit of the large-argument series (its terms grow like
// (v^2 / 2x)^k / k!) and needs no logarithm.
// Threshold compares of non-negative doubles on their bit patterns (same
// order as the values; integer instructions).
#define LB_GT(a, c) (__double_as_longlong(a) > __double_as_longlong(c))
#define LB_LT(a, c) (__double_as_longlong(a) < __double_as_longlong(c))
#define LB_GE(a, c) (!LB_LT(a, c))
#define LB_LE(a, c) (!LB_GT(a, c))
// A double cut (truncated) to single precision from its bit fields (signed
// 0 below 2^-126, signed inf from 2^128 up; NaN not expected): integer
// instructions, no FP64 conversion instruction.  For the single-precision
// estimates (edges, term counts) of the FP64 expressions.
__device__ __forceinline__ float f32_cut(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -126) return __uint_as_float(sgn);
  if (e > 127) return __uint_as_float(sgn | 0x7f800000u);
  return __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}
// The curved edge v^2 < 3.24 x in single precision: it moves the edge by at
// most a few 1e-7 relative, where the truncation error of mu_20 changes by
// as little, and spares every pair three FP64 instructions.
__device__ __forceinline__ bool tight_mu20(double v, double x) {
  if (LB_GT(x, 30.0) && LB_LT(v, 13.6)) return true;
  if (!LB_GT(x, 59.6925)) return false;
  const float vf = f32_cut(v);
  return vf * vf < 3.24f * f32_cut(x);
}
__device__ __forceinline__ bool tight_u13(double v, double x) { return (LB_GT(x, 25.0) && LB_GT(v, 0.7)) || LB_GT(v, 16.0); }

// Values (not the x-derivatives) take mu_20 and U_13 further into the
// fallback region than the shared thresholds: the truncation error of both
// expansions, measured the same way for each function (exact arithmetic of
// the truncated sums against the oracle, 1500 random points per added
// range, half of them at its edges), stays at or below 3.1e-16 of the error
// scale in
//   log K:  mu_20  x > 18.5, v < 9.5;  x > 20, v < 12.5;  x > 22, v < 13.6
//           U_13   x > 19, v > 10;     x > 14, v > 14
//   log I:  mu_20  x > 19, v < 4.5;    x > 21, v < 7.5;   x > 23, v < 9.5
//           U_13   x > 19.5, v > 10;   x > 17.5, v > 12;  x > 14.5, v > 14
// (log I's mu_20 converges more slowly as v^2/x grows: up to 1e-13 inside
// log K's ranges).  Pairs of these ranges leave the power series and the K
// integral, the costliest expressions.
enum WideRanges { WIDE_NONE = 0, WIDE_I = 1, WIDE_K = 2 };
__device__ __forceinline__ bool tight_mu20_w(double v, double x, int w) {
  if (tight_mu20(v, x)) return true;
  if (w == WIDE_K)
    return (LB_GT(x, 18.5) && LB_LT(v, 9.5)) || (LB_GT(x, 20.0) && LB_LT(v, 12.5)) ||
           (LB_GT(x, 22.0) && LB_LT(v, 13.6));
  if (w == WIDE_I)
    return (LB_GT(x, 19.0) && LB_LT(v, 4.5)) || (LB_GT(x, 21.0) && LB_LT(v, 7.5)) ||
           (LB_GT(x, 23.0) && LB_LT(v, 9.5));
  return false;
}
__device__ __forceinline__ bool tight_u13_w(double v, double x, int w) {
  if (tight_u13(v, x)) return true;
  if (w == WIDE_K) return (LB_GT(x, 19.0) && LB_GT(v, 10.0)) || (LB_GT(x, 14.0) && LB_GT(v, 14.0));
  if (w == WIDE_I)
    return (LB_GT(x, 19.5) && LB_GT(v, 10.0)) || (LB_GT(x, 17.5) && LB_GT(v, 12.0)) ||
           (LB_GT(x, 14.5) && LB_GT(v, 14.0));
  return false;
}

// With the pairs binned per expression on chip (no warp divergence), the
// tight dispatch also uses the shorter uniform expansions of the paper's CPU
// order, with order thresholds from the same error map: U_4 for v > 230,
// U_6 for v > 70, U_9 for v > 28 (truncation <= 2e-16 for every x).
// w: WIDE_I or WIDE_K for values of log I or log K (K callers pass |v|),
// which take the wider mu_20 and U_13 ranges above; WIDE_NONE for the
// x-derivatives.
__device__ __forceinline__ int classify(double v, double x, int mode, int w = WIDE_NONE) {
  if (mode == MODE_TIGHT) {
    if (tight_mu20_w(v, x, w)) return R_MU20;
    if (LB_GT(v, 230.0)) return R_U4;
    if (LB_GT(v, 70.0)) return R_U6;
    if (LB_GT(v, 28.0)) return R_U9;
    if (tight_u13_w(v, x, w)) return R_U13;
    return R_FALLBACK;
  }
  if (mode == MODE_PAPER_CPU) {
    if (paper_mu3(v, x)) return R_MU3;
    if (paper_mu20(v, x)) return R_MU20;
    if (paper_u4(v, x)) return R_U4;
    if (paper_u6(v, x)) return R_U6;
    if (paper_u9(v, x)) return R_U9;
    if (paper_u13(v, x)) return R_U13;
    return R_FALLBACK;
  }
  if (paper_mu20(v, x)) return R_MU20;
  if (paper_u13(v, x)) return R_U13;
  return R_FALLBACK;
}

// ---------------------------------------------------------------------------
// mu_K expression (K terms after the leading 1):
//   S = 1 + sum_{k=1}^{K} s^k prod_{j<=k} (mu - (2j-1)^2) / (k! (8x)^k),  mu = 4v^2
//   log I = x - log(2 pi x)/2 + log|S|          (s = -1)
//   log K = log(pi / (2x))/2 - x + log|S|       (s = +1)
// S is formed by Horner's rule on the term ratios
//   r_k = (mu - (2k-1)^2) / (8 x k),  S = 1 + s r_1 (1 + s r_2 (1 + ... (1 + s r_K))).
// ---------------------------------------------------------------------------
// The number of terms actually summed is the smallest n <= K after which
// the terms fall below 2^-56 (a later term is then below the rounding of S),
// found with a single-precision pass (mu_terms) and made uniform across the
// warp, so the double-precision Horner loop never diverges.  The tile kernel
// estimates n while it bins the pairs and orders each region by it, so the
// warps' lanes need similar counts.
template <int K>
__device__ __forceinline__ int mu_terms(float v, float x) {
  int n = K;
  // unrolled, so (2k-1)^2 and 1/k are constants: no division, no branch
  const float muf = 4.0f * v * v, inv8xf = __fdividef(1.0f, 8.0f * x);
  float t = 1.0f;
  bool found = false;
#pragma unroll
  for (int k = 1; k <= K; ++k) {
    t *= (muf - (float)((2 * k - 1) * (2 * k - 1))) * (inv8xf * (1.0f / (float)k));
    const bool hit = !found && fabsf(t) < 1.4e-17f;
    n = hit ? k : n;
    found = found || hit;
  }
  return n;
}

// Terms of the power series of log I (series_log_i, series_so): the count
// n after which a term falls below 2^-56 of the running sum past the peak
// index (Eq. "K"), by a single-precision pass; at most 90.  Returned packed
// with the number h of leading terms kept in FP64: the terms past the peak
// from the first one below 1e-4 of the running sum on are summed in
// double-float (their part of the sum is below 1e-3 of it), as
// n + 128 h (series_count, series_head unpack it).
__device__ __forceinline__ int series_terms(float v, float x) {
  int n = 1, h = 0;
  const float yf = 0.25f * x * x;
  const float kpk = 0.5f * (sqrtf(fmaf(x, x, v * v)) - v);
  float term = 1.0f, T = 0.0f, kf = 0.0f;
#pragma unroll 1
  for (int k = 1; k <= 90; ++k) {
    kf += 1.0f;
    term *= __fdividef(yf, kf * (kf + v));         // an estimate: the fast division suffices
    T += term;
    n = k;
    if (h == 0 && kf > kpk && term <= 1e-4f * (1.0f + T)) h = k;
    if (kf > kpk && term <= 1.4e-17f * (1.0f + T)) break;
  }
  return n + 128 * (h == 0 ? n : h);
}
__device__ __forceinline__ int series_count(int packed) { return packed & 127; }
__device__ __forceinline__ int series_head(int packed) { return packed >> 7; }

// Leading terms of mu_K kept in FP64: the smallest k at which the running
// product of the term ratios (the k-th term against the leading 1) falls
// below 1e-3, by the single-precision pass of mu_terms; K when none does.
// The terms past it hold less than 1e-3 of the sum and are summed in
// double-float (relative error a few 2^-48, below 1e-17 of the sum).
template <int K>
__device__ __forceinline__ int mu_head(float v, float x) {
  int m = K;
  const float muf = 4.0f * v * v, inv8xf = __fdividef(1.0f, 8.0f * x);
  float t = 1.0f;
  bool found = false;
#pragma unroll
  for (int k = 1; k <= K; ++k) {
    t *= (muf - (float)((2 * k - 1) * (2 * k - 1))) * (inv8xf * (1.0f / (float)k));
    const bool hit = !found && fabsf(t) < 1e-3f;
    m = hit ? k : m;
    found = found || hit;
  }
  return m;
}

// 1/k and (2k-1)^2/k for k = 1..20, the constants of the term ratios of
// mu_K, for a rolled loop over the warp's own number of terms (entry 0
// unused).  A fully unrolled loop with the terms above n switched off by a
// predicate would still issue every term's FP64 instructions.
static __constant__ double kMuInvK[21] = {0.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0, 1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0, 1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0, 1.0 / 19.0, 1.0 / 20.0};
static __constant__ double kMuOddK[21] = {0.0, 1.0 / 1.0, 9.0 / 2.0, 25.0 / 3.0, 49.0 / 4.0, 81.0 / 5.0, 121.0 / 6.0, 169.0 / 7.0, 225.0 / 8.0, 289.0 / 9.0, 361.0 / 10.0, 441.0 / 11.0, 529.0 / 12.0, 625.0 / 13.0, 729.0 / 14.0, 841.0 / 15.0, 961.0 / 16.0, 1089.0 / 17.0, 1225.0 / 18.0, 1369.0 / 19.0, 1521.0 / 20.0};
// 1/k as pairs of floats hi + lo (hi = 1/k rounded to single precision, lo
// the rest), for the double-float terms.
static __constant__ float kMuInvKh[21] = {0.0f, 0x1.p+0f, 0x1.p-1f, 0x1.555556p-2f, 0x1.p-2f, 0x1.99999ap-3f, 0x1.555556p-3f, 0x1.24924ap-3f, 0x1.p-3f, 0x1.c71c72p-4f, 0x1.99999ap-4f, 0x1.745d18p-4f, 0x1.555556p-4f, 0x1.3b13b2p-4f, 0x1.24924ap-4f, 0x1.111112p-4f, 0x1.p-4f, 0x1.e1e1e2p-5f, 0x1.c71c72p-5f, 0x1.af286cp-5f, 0x1.99999ap-5f};
static __constant__ float kMuInvKl[21] = {0.0f, 0.0f, 0.0f, -0x1.555556p-27f, 0.0f, -0x1.99999ap-29f, -0x1.555556p-28f, -0x1.b6db6ep-28f, 0.0f, -0x1.c71c72p-31f, -0x1.99999ap-30f, -0x1.745d18p-29f, -0x1.555556p-29f, -0x1.89d89ep-29f, -0x1.b6db6ep-29f, -0x1.dddddep-29f, 0.0f, -0x1.e1e1e2p-33f, -0x1.c71c72p-32f, -0x1.af286cp-32f, -0x1.99999ap-31f};

// mu_K with the lane's term count n given (at most K); all 32 lanes of the
// warp call it together.
template <int KIND, int K>
__device__ __forceinline__ double mu_expr_n(double v, double x, int n) {
  n = __reduce_max_sync(0xffffffffu, n);
  const int h = __reduce_max_sync(0xffffffffu, mu_head<K>(f32_cut(v), f32_cut(x)));
  const double mu = 4.0 * v * v;
  const double rx = ix_rcp_call(8.0 * x);                             // 1/(8x) on the integer pipe
  const double inv8x = (KIND == KIND_I) ? -rx : rx;                   // the sign s folded in
  double P = 1.0;
  int top = n;
  if (n > h) {
    // terms h+1..n in double-float: r_k = (mu s/(8x) - (2k-1)^2 s/(8x)) / k,
    // P <- 1 + r_k P
    const dfloat wd = df_from_double(inv8x), muw = df_from_double(mu * inv8x);
    dfloat Pd = df_make(1.0f, 0.0f);
#pragma unroll 1
    for (int k = n; k > h; --k) {
      const float odd = (float)((2 * k - 1) * (2 * k - 1));           // exact
      const dfloat ow = df_mul(wd, df_make(-odd, 0.0f));
      const dfloat r = df_mul(df_add(muw, ow), df_make(kMuInvKh[k], kMuInvKl[k]));
      Pd = df_mul_add(r, Pd, df_make(1.0f, 0.0f));
    }
    P = df_to_double(Pd);
    top = h;
  }
  // Three FP64 operations per leading term: a = mu/k - (2k-1)^2/k,
  // P = 1 + (a s/(8x)) P, for the warp's leading terms only.
#pragma unroll 1
  for (int k = top; k >= 1; --k) {
    const double a = fma(mu, kMuInvK[k], -kMuOddK[k]);
    P = fma(a * inv8x, P, 1.0);
  }
  // log(S / sqrt(2 pi x)) = log(S^2 / (2 pi x)) / 2 and
  // log(S sqrt(pi / (2x))) = log(S^2 pi / (2x)) / 2, with 1/x = 8 |inv8x|:
  // no square root needed.
  const double S2 = P * P;
  if (KIND == KIND_I) return fma(0.5, ix_log_call(S2 * rx * (8.0 / kTwoPi)), x);   // rx = |inv8x|
  return fma(0.5, ix_log_call(S2 * rx * (4.0 * kPi)), -x);
}

template <int KIND, int K>
__device__ __forceinline__ double mu_expr(double v, double x) {
  return mu_expr_n<KIND, K>(v, x, mu_terms<K>(f32_cut(v), f32_cut(x)));
}

// P_k(p) of the Debye polynomial u_k(t) = t^k P_k(t^2); k is a compile-time
// constant after unrolling, so the switch folds away.
template <typename T>
__device__ __forceinline__ T debye_P(int k, T p) {
  switch (k) {
    case 1: return lb_debye_P1(p);
    case 2: return lb_debye_P2(p);
    case 3: return lb_debye_P3(p);
    case 4: return lb_debye_P4(p);
    case 5: return lb_debye_P5(p);
    case 6: return lb_debye_P6(p);
    case 7: return lb_debye_P7(p);
    case 8: return lb_debye_P8(p);
    case 9: return lb_debye_P9(p);
    case 10: return lb_debye_P10(p);
    case 11: return lb_debye_P11(p);
    case 12: return lb_debye_P12(p);
    default: return lb_debye_P13(p);
  }
}

// P_k(p) in double-float, k = 2..13 (warp-uniform), by a rolled Horner
// loop over the coefficient pairs of lb_debye_df (constant memory, read by
// all lanes at once): the unrolled sums of U_13 alone would be about 1500
// instructions, and the tile kernel's warps run several expressions at a
// time out of one instruction cache.
__device__ __forceinline__ dfloat debye_P_df(int k, dfloat p) {
  const float(*c)[2] = lb_debye_df + lb_debye_df_off[k];
  dfloat r = df_make(c[k][0], c[k][1]);
#pragma unroll 1
  for (int i = k - 1; i >= 0; --i) r = df_mul_add(r, p, df_make(c[i][0], c[i][1]));
  return r;
}

// Q_k(p) in double-float, k = 2..13, from lb_debye_qdf (same layout).
__device__ __forceinline__ dfloat debye_Q_df(int k, dfloat p) {
  const float(*c)[2] = lb_debye_qdf + lb_debye_df_off[k];
  dfloat r = df_make(c[k][0], c[k][1]);
#pragma unroll 1
  for (int i = k - 1; i >= 0; --i) r = df_mul_add(r, p, df_make(c[i][0], c[i][1]));
  return r;
}

template <typename T>
__device__ __forceinline__ T debye_Q(int k, T p) {
  switch (k) {
    case 1: return lb_debye_Q1(p);
    case 2: return lb_debye_Q2(p);
    case 3: return lb_debye_Q3(p);
    case 4: return lb_debye_Q4(p);
    case 5: return lb_debye_Q5(p);
    case 6: return lb_debye_Q6(p);
    case 7: return lb_debye_Q7(p);
    case 8: return lb_debye_Q8(p);
    case 9: return lb_debye_Q9(p);
    case 10: return lb_debye_Q10(p);
    case 11: return lb_debye_Q11(p);
    case 12: return lb_debye_Q12(p);
    default: return lb_debye_Q13(p);
  }
}

// ---------------------------------------------------------------------------
// U_K expression (paper Eqs. "log Iv u k", "log Kv u k"):
//   x' = x/v, r = sqrt(1 + x'^2), t = 1/r, eta = r + log(x' / (1 + r)),
//   S = 1 + sum_{k=1}^{K} (+-1)^k u_k(t) / v^k  (+ for I, alternating for K)
//   log I = -log(2 pi v)/2 + v eta - log(1 + x'^2)/4 + log|S|
//   log K =  log(pi/(2v))/2 - v eta - log(1 + x'^2)/4 + log|S|
// with u_k(t) = t^k P_k(t^2) (Debye polynomials, generated exactly from the
// recurrence of Eqs. "u0", "uk").  The two log terms are merged:
// -log(2 pi v)/2 - log(r)/2 = log(1 / sqrt(2 pi v r)).
// ---------------------------------------------------------------------------
template <int KIND, int K>
__device__ __forceinline__ double u_expr(double v, double x) {
  const double inv_v = ix_rcp_call(v);           // reciprocal and root on the integer pipe
  const double xp = x * inv_v;
  double r, t;
  if (LB_LT(xp, 1e150)) {
    const double r2 = fma(xp, xp, 1.0);
    t = ix_rsqrt_call(r2);                       // t = (1 + x'^2)^-1/2
    r = r2 * t;
  } else {
    r = xp;                                      // 1 + x'^2 rounds to x'^2
    t = ix_rcp_call(r);
  }
  const double p = t * t;
  const double tq = t * inv_v;                    // t / v
  const double q = (KIND == KIND_K) ? -tq : tq;
  // Horner in q over k = K..1:  S = 1 + q (P_1 + q (P_2 + ... + q P_K)).
  // The terms k >= 2 (at most 1/v^2 of the sum, with v > 0.7 and x' > 35 or
  // v > 16 in the U regions: below 1e-3 of it) in double-float, P_1 and the
  // two outer steps in FP64.
  const dfloat pd = df_from_double(p), qd = df_from_double(q);
  dfloat accd = debye_P_df(K, pd);
#pragma unroll 1
  for (int k = K - 1; k >= 2; --k) accd = df_mul_add(accd, qd, debye_P_df(k, pd));
  const double acc = fma(df_to_double(accd), q, lb_debye_P1(p));
  const double S = fma(acc, q, 1.0);
  const double eta = r + (ix_log_call(xp) - ix_log_call(1.0 + r));      // log(x' / (1 + r)), no division
  // log(S / sqrt(2 pi v r)) = log(S^2 t / v) / 2 - log(2 pi) / 2, and for K
  // log(S sqrt(pi / (2 v r))) = log(S^2 t / v) / 2 + log(pi / 2) / 2
  // (t = 1/r): no root, and the constant joins the FMA with v eta.
  const double w = S * S * tq;
  if (KIND == KIND_I) return fma(0.5, ix_log_call(w), fma(v, eta, -kHalfLog2Pi));
  return fma(0.5, ix_log_call(w), fma(-v, eta, kHalfLogHalfPi));
}

// ---------------------------------------------------------------------------
// Power series of I_v (fallback region of log I):
//   a_0 = 1/Gamma(v+1), a_{k+1} = a_k x^2 / (4 (k+1)(k+v+1))      (Eq. "ak recurrence")
//   log I_v(x) = v log(x/2) + log a_0 + log sum_k a_k / a_0       (Eq. "log Iv")
// The log-sum-exp shift is a_0 instead of the peak term a_K: any shift is
// exact, and in the fallback region (x <= 30) the largest ratio a_K/a_0 is
// below e^x, far from overflow, so the terms can be summed in linear scale
// without a logarithm per term.  Terms are kept until they fall below 2^-56
// of the running sum after the peak index K = (-v + sqrt(x^2 + v^2))/2
// (Eq. "K"), the truncation rule of Sec. 3.1; the count n is found with a
// single-precision pass and made uniform across the warp.  The sum
//   S = 1 + r_1 (1 + r_2 (1 + ... (1 + r_n))),  r_k = y / (k (k + v)),  y = x^2/4,
// is then evaluated backwards as a fraction A/B (A <- d_k B + y A,
// B <- d_k B with d_k = k (k + v)), so the double-precision loop has no
// division; B stays below 1e250 for n <= 80 and v <= 16.  All 32 lanes of the
// warp must call it together.
// ---------------------------------------------------------------------------
// k and k^2 for k = 0, 1, ..., 90 as doubles (exact): the series loop reads
// them from constant memory (k is warp-uniform) and forms d_k = k (k + v) as
// one FMA, k v + k^2, instead of an addition and a multiplication.
static __constant__ double kSeriesK[91] = {
    0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25,
    26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 46, 47, 48, 49,
    50, 51, 52, 53, 54, 55, 56, 57, 58, 59, 60, 61, 62, 63, 64, 65, 66, 67, 68, 69, 70, 71, 72, 73,
    74, 75, 76, 77, 78, 79, 80, 81, 82, 83, 84, 85, 86, 87, 88, 89, 90};
static __constant__ double kSeriesK2[91] = {
    0, 1, 4, 9, 16, 25, 36, 49, 64, 81, 100, 121, 144, 169, 196, 225, 256, 289, 324, 361, 400, 441,
    484, 529, 576, 625, 676, 729, 784, 841, 900, 961, 1024, 1089, 1156, 1225, 1296, 1369, 1444,
    1521, 1600, 1681, 1764, 1849, 1936, 2025, 2116, 2209, 2304, 2401, 2500, 2601, 2704, 2809, 2916,
    3025, 3136, 3249, 3364, 3481, 3600, 3721, 3844, 3969, 4096, 4225, 4356, 4489, 4624, 4761, 4900,
    5041, 5184, 5329, 5476, 5625, 5776, 5929, 6084, 6241, 6400, 6561, 6724, 6889, 7056, 7225, 7396,
    7569, 7744, 7921, 8100};

// y / (k (k + v)) in double-float: the denominator from k v + k^2 (k^2
// exact), the quotient as q1 + q2 (Dekker: q1 from the leading parts, q2
// from the remainder y - q1 d).
__device__ __forceinline__ dfloat series_ratio_df(dfloat y, dfloat v, int k) {
  const float kf = (float)k;
  const dfloat d = df_add(df_mul(v, df_make(kf, 0.0f)), df_make(kf * kf, 0.0f));
  const float q1 = y.h * __frcp_rn(d.h);
  const dfloat rem = df_add(y, df_mul(d, df_make(-q1, 0.0f)));
  const float q2 = rem.h * __frcp_rn(d.h);
  dfloat r;
  r.h = q1 + q2;
  r.l = q2 - (r.h - q1);
  return r;
}

__device__ __forceinline__ double series_log_i_n(double v, double x, int packed) {
  const int n = __reduce_max_sync(0xffffffffu, series_count(packed));
  const int h = __reduce_max_sync(0xffffffffu, series_head(packed));
  const double y = 0.25 * x * x;
  double A = 1.0, B = 1.0;
  int top = n;
  if (n > h) {
    // terms h+1..n: P <- 1 + (y / (k (k + v))) P in double-float; its value
    // then starts the FP64 fraction (A / B = P)
    const dfloat yd = df_from_double(y), vd = df_from_double(v);
    dfloat Pd = df_make(1.0f, 0.0f);
#pragma unroll 1
    for (int k = n; k > h; --k) Pd = df_mul_add(series_ratio_df(yd, vd, k), Pd, df_make(1.0f, 0.0f));
    A = df_to_double(Pd);
    top = h;
  }
#pragma unroll 1
  for (int k = top; k >= 1; --k) {
    const double d = fma(kSeriesK[k], v, kSeriesK2[k]);   // k (k + v), exact up to one rounding
    A = fma(d, B, y * A);
    B *= d;
  }
  double res = ix_log_call(A * ix_rcp_call(B)) - lgamma(v + 1.0);
  if ((__double_as_longlong(v) << 1) != 0) res = fma(v, ix_log_call(0.5 * x), res);   // v != 0, on the bits
  return res;
}

__device__ __forceinline__ double series_log_i(double v, double x) {
  return series_log_i_n(v, x, series_terms(f32_cut(v), f32_cut(x)));
}

// ---------------------------------------------------------------------------
// One order for every argument (v_stride 0).  The order-dependent parts of
// the expressions are then the same for every pair, and a block computes
// them once (scalar_order_setup):
//   mu_K:   S = sum_k a_k w^k, w = 1/(8x), a_k = s^k prod_{j<=k} (mu - (2j-1)^2) / k!
//           -- one FMA per term instead of three;
//   series: P <- 1 + (y / (k (k + v))) P with the reciprocals 1/(k (k + v))
//           tabulated -- two operations per term instead of six, and
//           lgamma(v + 1) once;
//   U_K:    S(t) = 1 + sum_k (s/v)^k u_k(t) = sum_m C_m t^m as one polynomial
//           of degree 3K in t -- 3K FMAs instead of K(K+3)/2, and 1/v once.
// The sums are the same sums in another order of operations.
// ---------------------------------------------------------------------------
struct ScalarOrder {
  double v, inv_v, lg1;                 // v, 1/v, lgamma(v + 1)
  double sig;                           // sigma: a power of two near mu/8 (1 for mu < 8)
  double mu[21];                        // a_0..a_20 / sigma^k (sign s of the kind folded in)
  double ser[91];                       // 1 / (k (k + v)), k = 1..90
  double u4[4], u6[4], u9[4], u13[4];   // C_0..C_3 of U_K
  dfloat mud[21];                       // mu[] in double-float
  dfloat serd[91];                      // ser[] in double-float
  dfloat u4d[13], u6d[19], u9d[28], u13d[40];   // C_0..C_3K in double-float (C_4.. used)
};

// All threads of the block call it; ends with a barrier.
template <int KIND>
__device__ __forceinline__ void scalar_order_setup(ScalarOrder& so, double v) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    so.v = v;
    so.inv_v = 1.0 / v;
    so.lg1 = lgamma(v + 1.0);
    const double mu = 4.0 * v * v, s = KIND == KIND_I ? -1.0 : 1.0;
    // a_k w^k = (a_k / sigma^k) (sigma w)^k: with sigma near mu/8 the scaled
    // coefficients stay below 8^k / k! (the unscaled ones overflow for
    // orders above about 1e9, and the double-float ones above 1e38)
    int j = 0;
    if (mu >= 16.0) j = ilogb(mu) - 3;
    so.sig = ldexp(1.0, j);
    double a = 1.0;
    so.mu[0] = 1.0;
    so.mud[0] = df_make(1.0f, 0.0f);
    for (int k = 1; k <= 20; ++k) {
      a = ldexp(a * (s * (mu - (double)((2 * k - 1) * (2 * k - 1)))) / (double)k, -j);
      so.mu[k] = a;
      so.mud[k] = df_from_double(a);
    }
  } else if (tid <= 90) {
    so.ser[tid] = 1.0 / ((double)tid * ((double)tid + v));
    so.serd[tid] = df_from_double(so.ser[tid]);
  } else if (tid >= 128 && tid < 228) {
    // C_m of U_K: the coefficients of t^m, sum over k + 2i = m of c_{k,i} (s/v)^k
    int j = tid - 128, K, m;
    double* dst;
    dfloat* dstd;
    if (j < 13) { K = 4; m = j; dst = so.u4; dstd = so.u4d; }
    else if (j < 32) { K = 6; m = j - 13; dst = so.u6; dstd = so.u6d; }
    else if (j < 60) { K = 9; m = j - 32; dst = so.u9; dstd = so.u9d; }
    else { K = 13; m = j - 60; dst = so.u13; dstd = so.u13d; }
    const double sv = (KIND == KIND_I ? 1.0 : -1.0) / v;
    double c = 0.0, pk = 1.0;
    for (int k = 0; k <= K; ++k) {
      if (k > 0) pk *= sv;
      const int twoi = m - k;
      if (twoi >= 0 && (twoi & 1) == 0 && (twoi >> 1) <= k) c = fma(lb_debye_c[k][twoi >> 1], pk, c);
    }
    if (m < 4) dst[m] = c;
    dstd[m] = df_from_double(c);
  }
  __syncthreads();
}

template <int KIND>
__device__ __forceinline__ double mu_expr_so(const ScalarOrder& so, double x, int n) {
  n = __reduce_max_sync(0xffffffffu, n);
  const int h = __reduce_max_sync(0xffffffffu, mu_head<20>(f32_cut(so.v), f32_cut(x)));
  const double w = ix_rcp_call(8.0 * x);
  const double ws = w * so.sig;                   // exact: sigma is a power of two
  double P = 0.0;
  int top = n;
  if (n > h) {                                    // terms h+1..n in double-float
    const dfloat wd = df_from_double(ws);
    dfloat Pd = so.mud[n];
#pragma unroll 1
    for (int k = n - 1; k > h; --k) Pd = df_mul_add(Pd, wd, so.mud[k]);
    P = df_to_double(Pd);
    top = h;
  }
#pragma unroll 1
  for (int k = top; k >= 0; --k) P = fma(P, ws, so.mu[k]);   // the warp's leading terms
  const double S2 = P * P;
  if (KIND == KIND_I) return fma(0.5, ix_log_call(S2 * w * (8.0 / kTwoPi)), x);
  return fma(0.5, ix_log_call(S2 * w * (4.0 * kPi)), -x);
}

template <int KIND, int K>
__device__ __forceinline__ double u_expr_so(const ScalarOrder& so, double x) {
  const double v = so.v, inv_v = so.inv_v;
  const double xp = x * inv_v;
  double r, t;
  if (LB_LT(xp, 1e150)) {
    const double r2 = fma(xp, xp, 1.0);
    t = ix_rsqrt_call(r2);
    r = r2 * t;
  } else {
    r = xp;
    t = ix_rcp_call(r);
  }
  const double* C = K == 4 ? so.u4 : (K == 6 ? so.u6 : (K == 9 ? so.u9 : so.u13));
  const dfloat* Cd = K == 4 ? so.u4d : (K == 6 ? so.u6d : (K == 9 ? so.u9d : so.u13d));
  // S = sum_m C_m t^m.  C_m for m >= 4 holds the parts of u_k, k >= 2 only
  // (u_k has the powers t^k .. t^3k), at most about 2e-3 of the sum in the
  // U regions: those terms in double-float, C_3 .. C_0 in FP64.
  const dfloat td = df_from_double(t);
  dfloat Sd = Cd[3 * K];
#pragma unroll 1
  for (int m = 3 * K - 1; m >= 4; --m) Sd = df_mul_add(Sd, td, Cd[m]);
  double S = df_to_double(Sd);
#pragma unroll
  for (int m = 3; m >= 0; --m) S = fma(S, t, C[m]);
  const double eta = r + (ix_log_call(xp) - ix_log_call(1.0 + r));
  const double w = S * S * (t * inv_v);          // as in u_expr
  if (KIND == KIND_I) return fma(0.5, ix_log_call(w), fma(v, eta, -kHalfLog2Pi));
  return fma(0.5, ix_log_call(w), fma(-v, eta, kHalfLogHalfPi));
}

__device__ __forceinline__ double series_so(const ScalarOrder& so, double x, int packed) {
  const double v = so.v;
  const int n = __reduce_max_sync(0xffffffffu, series_count(packed));
  const int h = __reduce_max_sync(0xffffffffu, series_head(packed));
  const double y = 0.25 * x * x;
  double P = 1.0;
  int top = n;
  if (n > h) {                                    // terms h+1..n in double-float
    const dfloat yd = df_from_double(y);
    dfloat Pd = df_make(1.0f, 0.0f);
#pragma unroll 1
    for (int k = n; k > h; --k) Pd = df_mul_add(df_mul(yd, so.serd[k]), Pd, df_make(1.0f, 0.0f));
    P = df_to_double(Pd);
    top = h;
  }
#pragma unroll 1
  for (int k = top; k >= 1; --k) P = fma(y * so.ser[k], P, 1.0);
  double res = ix_log_call(P) - so.lg1;
  if ((__double_as_longlong(v) << 1) != 0) res = fma(v, ix_log_call(0.5 * x), res);   // v != 0, on the bits
  return res;
}

// ---------------------------------------------------------------------------
// x-derivatives of the same expressions (the adjoint of the forward path).
// Each differentiates its expression term by term, so it is valid exactly
// where the expression is; the paper lists derivatives as future work
// (Sec. 7), and these follow directly from its Eqs.
// ---------------------------------------------------------------------------

// mu_K: log f = +-x - log(2 pi x)/2 + log S (I: +x, K: -x and +log(pi/2)/2),
// S = 1 + sum_k c_k x^-k, so d/dx log f = +-1 - 1/(2x) - (sum_k k c_k x^-k) / (x S).
template <int KIND, int K>
__device__ __forceinline__ double mu_dx(double v, double x) {
  const double mu = 4.0 * v * v;
  const double inv8x = ix_rcp(8.0 * x);             // the reciprocals on the integer pipe
  double term = 1.0, S = 1.0, D = 0.0;
#pragma unroll
  for (int k = 1; k <= K; ++k) {
    const double odd = (double)((2 * k - 1) * (2 * k - 1));
    double r = (mu - odd) * (inv8x * (1.0 / (double)k));
    if (KIND == KIND_I) r = -r;
    term *= r;
    S += term;
    D = fma((double)k, term, D);
  }
  const double inv_x = 8.0 * inv8x;                 // exact scaling
  const double base = (KIND == KIND_I) ? 1.0 : -1.0;
  return base - inv_x * fma(D, ix_rcp(S), 0.5);
}

// The same for the first n terms only (n: the pair's term count, made
// warp-uniform), as a rolled loop: the terms past n are below 2^-56 of S.
template <int KIND, int K>
__device__ __forceinline__ double mu_dx_n(double v, double x, int n) {
  n = __reduce_max_sync(0xffffffffu, n);
  const double mu = 4.0 * v * v;
  const double rx = ix_rcp(8.0 * x);                // on the integer pipe
  const double inv8x = (KIND == KIND_I) ? -rx : rx;  // the sign folded in
  double term = 1.0, S = 1.0, D = 0.0, kd = 0.0;
#pragma unroll 1
  for (int k = 1; k <= n; ++k) {
    kd += 1.0;
    term *= fma(mu, kMuInvK[k], -kMuOddK[k]) * inv8x;
    S += term;
    D = fma(kd, term, D);
  }
  const double base = (KIND == KIND_I) ? 1.0 : -1.0;
  return base - (8.0 * rx) * fma(D, ix_rcp(S), 0.5);
}

// U_K: with x' = x/v, t = (1 + x'^2)^-1/2, d(v eta)/dx = 1/(t x'),
// d/dx [-log(1 + x'^2)/4] = -x' t^2 / (2v), dt/dx = -x' t^3 / v and
// d/dt u_k(t) = t^(k-1) Q_k(t^2):
//   d/dx log f = +-1/(t x') - (x' t^2 / v) (1/2 + SQ / S),
//   S = 1 + sum q^k P_k(t^2), SQ = sum q^k Q_k(t^2), q = +-t/v.
template <int KIND, int K>
__device__ __forceinline__ double u_dx(double v, double x) {
  const double inv_v = ix_rcp(v);                  // reciprocals and 1/sqrt on the integer pipe
  const double xp = x * inv_v;
  double r, t;
  if (xp < 1e150) {
    const double w = fma(xp, xp, 1.0);
    t = ix_rsqrt(w);
    r = w * t;
  } else {
    r = xp;
    t = ix_rcp(xp);
  }
  const double p = t * t;
  double q = t * inv_v;
  if (KIND == KIND_K) q = -q;
  // Horner in q over k = K..1 for S and SQ; as in u_expr, the terms k >= 2
  // (at most 1/v^2 of each sum in the U regions) in double-float, rolled
  // over the coefficient tables, and k = 1 and the outer steps in FP64.
  const dfloat pd = df_from_double(p), qd = df_from_double(q);
  dfloat aP = debye_P_df(K, pd), aQ = debye_Q_df(K, pd);
#pragma unroll 1
  for (int k = K - 1; k >= 2; --k) {
    aP = df_mul_add(aP, qd, debye_P_df(k, pd));
    aQ = df_mul_add(aQ, qd, debye_Q_df(k, pd));
  }
  const double accP = fma(df_to_double(aP), q, lb_debye_P1(p));
  const double accQ = fma(df_to_double(aQ), q, lb_debye_Q1(p));
  const double S = fma(accP, q, 1.0);
  const double SQ = accQ * q;
  const double lead = r * ix_rcp(xp);               // 1/(t x') = sqrt(1 + x'^2)/x'
  const double corr = (xp * p * inv_v) * fma(SQ, ix_rcp(S), 0.5);
  return (KIND == KIND_I) ? lead - corr : -lead - corr;
}

// Series: log I = v log(x/2) - lgamma(v+1) + log(1 + T), T = sum_{k>=1} a_k/a_0
// with a_k/a_0 proportional to x^(2k):  d/dx log I = v/x + (2/x) (sum k a_k/a_0) / (1 + T).
// With the pair's term count (series_terms): T and D = sum k a_k/a_0 by one
// backward Horner pass, P <- 1 + r_k P and E <- r_k (P + E) (E collects
// y dP/dy = D, as r_k is proportional to y), r_k = y / (k (k + v)); the
// terms past the head in double-float (as series_log_i_n), the head as one
// fraction P = A/B, E = C/B with A <- d B + y A, C <- y (A + C), B <- d B
// (d = k (k + v)), so no term divides; D/(1+T) = C/A.
__device__ __forceinline__ double series_dx_n(double v, double x, int packed) {
  const int n = __reduce_max_sync(0xffffffffu, series_count(packed));
  const int h = __reduce_max_sync(0xffffffffu, series_head(packed));
  const double y = 0.25 * x * x;
  double A = 1.0, C = 0.0, B = 1.0;
  int top = n;
  if (n > h) {
    const dfloat yd = df_from_double(y), vd = df_from_double(v);
    dfloat Pd = df_make(1.0f, 0.0f), Ed = df_make(0.0f, 0.0f);
#pragma unroll 1
    for (int k = n; k > h; --k) {
      const dfloat r = series_ratio_df(yd, vd, k);
      Ed = df_mul(r, df_add(Pd, Ed));
      Pd = df_mul_add(r, Pd, df_make(1.0f, 0.0f));
    }
    A = df_to_double(Pd);
    C = df_to_double(Ed);
    top = h;
  }
#pragma unroll 1
  for (int k = top; k >= 1; --k) {
    const double d = fma(kSeriesK[k], v, kSeriesK2[k]);   // k (k + v)
    C = y * (A + C);
    A = fma(d, B, y * A);
    B *= d;
  }
  return fma(2.0 * C, ix_rcp(A), v) * ix_rcp(x);
}

}  // namespace lb
