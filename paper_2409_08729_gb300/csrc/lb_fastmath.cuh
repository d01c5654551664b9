// lb_fastmath.cuh -- double-precision exp and log with few FP64 operations.
//
// On GB300 the FP64 pipe issues one warp instruction per 16 cycles per SM
// (1/62 of FP32), and the log-Bessel kernels spend most of it in exp and
// log.  These are table-driven implementations after P. T. P. Tang
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989; "... of the logarithm
// function ...", ACM TOMS 16(4), 1990): argument reduction with tables
// (gen_fastmath.py: 512 entries for exp, 128 for log), a short polynomial,
// and exponent handling with integer instructions, which run on other pipes.
// 10 (exp; 9 without the low table part) and 14 (log) FP64 operations per
// call.  Both fall back to the libm function
// outside their fast range (|y| >= 708 for exp; zero, negative, subnormal,
// infinite or NaN arguments for log).  Accuracy is checked against the
// double-double oracle and against CUDA's exp/log in the test suite.
#pragma once

#include "fastmath_tables.h"

namespace lb {

// Shared core of the exps: y = (k / 512) ln 2 + r, |r| <= ln2 / 1024, k split
// as 512 m + j; e^y = 2^m 2^(j/512) e^r.  Returns 2^(j/512) (1 + p) with
// p = e^r - 1 (|r|^5/120 < 1.2e-18 is the truncation of the degree-4
// polynomial); `lo` adds the low part of the table entry.  The caller
// applies 2^m to the exponent field (integer add).
template <bool LO>
__device__ __forceinline__ double fm_exp_core(double y, int* m) {
  const double shifter = 6755399441055744.0;                 // 1.5 * 2^52
  const double t = fma(y, LB_FM_INV_L, shifter);             // rint(y * 512 / ln 2) in the low bits
  const int k = __double2loint(t);
  const double kd = t - shifter;
  double r = fma(-kd, LB_FM_L_HI, y);                        // exact: kd * L_HI has <= 53 bits
  r = fma(-kd, LB_FM_L_LO, r);
  double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r * r, r);
  const int j = k & 511;
  *m = k >> 9;
  const double th = __ldg(lb_fm_exp_hi + j);
  return LO ? fma(th, p, __ldg(lb_fm_exp_lo + j)) + th : fma(th, p, th);
}

__device__ __forceinline__ double fm_exp(double y) {
  if (!(fabs(y) < 708.0)) return exp(y);
  int m;
  const double res = fm_exp_core<true>(y, &m);
  return __hiloint2double(__double2hiint(res) + (m << 20), __double2loint(res));
}

// exp(y) for y <= 708 (callers never pass more); y < -708 gives 0.  The range
// test and the flush use integer instructions only, so no FP64 compare is
// spent and there is no divergent fall-back path.
__device__ __forceinline__ double fm_exp_le(double y) {
  const bool under = (unsigned int)__double2hiint(y) > 0xC0862000u;     // y < -708 (sign bit set)
  if (under) y = -708.0;
  int m;
  const double res = fm_exp_core<true>(y, &m);
  const double out = __hiloint2double(__double2hiint(res) + (m << 20), __double2loint(res));
  return under ? 0.0 : out;
}

// fm_exp_le without the low table part: within about 1 ulp instead of 0.5,
// one FP64 operation less (for sums of many terms, where a 1-ulp error per
// term is far below the sum's own rounding).  The kernels now take their
// node exps from the integer pipes (lb_intmath.cuh); this one stays
// available and measured for comparison.
__device__ __forceinline__ double fm_exp_term(double y) {
  const bool under = (unsigned int)__double2hiint(y) > 0xC0862000u;
  if (under) y = -708.0;
  int m;
  const double res = fm_exp_core<false>(y, &m);
  const double out = __hiloint2double(__double2hiint(res) + (m << 20), __double2loint(res));
  return under ? 0.0 : out;
}

// Order-preserving map of a double to an int through its high word (larger
// double, larger key); key_to_double returns a double within 2^-20
// (relative) of the original.  Used for warp max reductions on the integer
// pipe: the maximum only serves as a log-sum-exp shift, where any nearby
// value is exact.
__device__ __forceinline__ int order_key(double a) {
  const int h = __double2hiint(a);
  return h >= 0 ? h : (h ^ 0x7fffffff);
}
__device__ __forceinline__ double key_to_double(int k) {
  const int h = k >= 0 ? k : (k ^ 0x7fffffff);
  return __hiloint2double(h, 0);
}

__device__ __forceinline__ double fm_log(double z) {
  const int hi = __double2hiint(z);
  const int lo = __double2loint(z);
  if (hi < 0x00100000 || hi >= 0x7ff00000) return log(z);   // <= 0 (sign bit), subnormal, inf, NaN
  const int j = (hi >> 13) & 127;                           // top 7 bits of the significand
  const int e = ((hi >> 20) - 1023) + (j >= LB_FM_LOG_JSPLIT ? 1 : 0);
  const double mant = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);   // in [1, 2)
  const double r = fma(mant, __ldg(lb_fm_log_c + j), -1.0);                   // |r| < 2^-7
  // log1p(r) = r - r^2 (1/2 - r (1/3 - r (1/4 - ... - r (1/7 - r/8))))
  // (truncation |r|^9/9 < 1.6e-18 |r|)
  double q = fma(r, -1.0 / 8.0, 1.0 / 7.0);
  q = fma(q, -r, 1.0 / 6.0);
  q = fma(q, -r, 1.0 / 5.0);
  q = fma(q, -r, 0.25);
  q = fma(q, -r, 1.0 / 3.0);
  q = fma(q, -r, 0.5);
  const double lp = fma(-r * r, q, r);
  // e as a double with one add: 2^52 + 2^31 + e, minus the offset
  const double ed = __hiloint2double(0x43300000, (int)(0x80000000u + (unsigned int)e)) - 4503601774854144.0;
  const double small = fma(ed, LB_FM_LN2_LO, __ldg(lb_fm_log_lo + j)) + lp;
  const double big = fma(ed, LB_FM_LN2_HI, __ldg(lb_fm_log_hi + j));        // exact product
  return big + small;
}

}  // namespace lb
