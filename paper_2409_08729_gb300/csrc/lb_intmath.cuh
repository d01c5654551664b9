// lb_intmath.cuh -- double-precision exp and log computed on the integer pipes.
//
// On GB300 the FP64 pipe retires 2 operations per SM per clock, while the
// integer pipes retire 64 each; a kernel whose FP64 work is mostly exp and
// log (the K integral: two exps and a log per quadrature node) is bound by
// the FP64 pipe with the integer pipes idle.  These versions follow the
// table-driven methods of P. T. P. Tang ("Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2),
// 1989; "... of the logarithm function ...", ACM TOMS 16(4), 1990) -- table
// reduction, a short polynomial, reconstruction -- but carry every step in
// 64- and 128-bit fixed-point integers (tables from gen_intmath.py), and
// build the double result from its bit fields.  No FP64 instruction is
// executed; ix_exp spends two FP32 instructions to estimate its reduction
// index.
//
//   ix_exp(y), y <= 708:  y = (k/512) ln2 + r, |r| <= 0.61 ln2/512, with k
//     estimated in single precision and r = y - k ln2/512 exact in Q116;
//     e^r - 1 by a degree-5 polynomial (inner steps in 32 bits, outer in
//     Q62, r in Q73); 2^(j/512)(1 + p) in Q62,
//     j = k mod 512; 2^(k div 512) into the exponent field.  Error below
//     0.51 ulp.  |y| < 2^-64 gives 1; y < -708 gives 0; y > 708 gives +inf.
//   ix_log(z), z positive and normal:  z = 2^e m, m in [1, 2); j = the top
//     9 fraction bits, r = m C_j / 2^13 - 1 exact (|r| < 2^-9.8; C_0 = 2^13
//     and C_511 = 2^12 keep arguments next to 1 exact), log(1 + r) by a
//     degree-6 polynomial, and e ln2 - log(C_j / 2^13) + log(1 + r) summed
//     in Q116 (128 bits): error below 0.51 ulp.  Other arguments (zero,
//     negative, subnormal, infinite, NaN) go to the libm log.
//   ix_log_q53, ix_mul_q58, ix_exp_q58_fx: the same methods between fixed-
//     point values (Q53 logarithms in, a Q58 exponential out), for sums of
//     e^(c + a log z - m) that never need the intermediate doubles.
//
// The functions are plain integer code: compiled for the host (without
// __CUDACC__) they give bit-identical results, which the CPU test suite
// checks against the oracle's double-double exp and log.
#pragma once

#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define LB_IX_FN __device__ __forceinline__
#define LB_IX_TABLE static __device__ const
#define LB_IX_LOAD(p) __ldg(p)
#else
#include <string.h>
#define LB_IX_FN static inline
#define LB_IX_TABLE static const
#define LB_IX_LOAD(p) (*(p))
#endif

#include "intmath_tables.h"

namespace lb {

LB_IX_FN int64_t ix_mulhi(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * (__int128)b) >> 64);
#endif
}

LB_IX_FN uint64_t ix_umulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

// high 32 bits of a 32 x 32-bit signed product
LB_IX_FN int32_t ix_mulhi32(int32_t a, int32_t b) {
#if defined(__CUDA_ARCH__)
  return __mulhi(a, b);
#else
  return (int32_t)(((int64_t)a * (int64_t)b) >> 32);
#endif
}

// floor(a b / 2^32) for a signed 64-bit a and a signed 32-bit b (|a b| < 2^95):
// two 32 x 32 -> 64-bit products instead of a 64 x 64 one.
LB_IX_FN int64_t ix_mul64x32hi(int64_t a, int32_t b) {
  const int64_t hi = (int64_t)(int32_t)(a >> 32) * (int64_t)b;
  const int64_t lo = (int64_t)((uint64_t)(uint32_t)a * (uint64_t)(int64_t)b);   // (a mod 2^32) b, exact in 64 bits
  return hi + (lo >> 32);
}

LB_IX_FN int ix_clz(uint64_t a) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)a);
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

LB_IX_FN uint64_t ix_bits(double d) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}

LB_IX_FN double ix_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

LB_IX_FN float ix_float(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __int_as_float((int)b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}

LB_IX_FN uint32_t ix_fbits(float f) {
#if defined(__CUDA_ARCH__)
  return (uint32_t)__float_as_int(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}

// 2^(j/512) (1 + p) in Q62 for y = (k/512) ln2 + r, r in Q73 (|r| < 2^-10.2),
// j = k mod 512, p = e^r - 1.
LB_IX_FN int64_t ix_exp_finish(int64_t r, int k) {
  // e^r - 1 = r (1 + r (1/2 + r (1/6 + r (1/24 + r/120)))).  The steps for
  // 1/24 and 1/6 enter the result times r^3 (|r| < 2^-10.2), so 32-bit
  // precision (Q31, r in Q41) suffices there; 1/2 and 1 are carried in Q62.
  const int32_t r32 = (int32_t)(r >> 32);                   // Q41
  int32_t a3 = LB_IX_E4 + (ix_mulhi32(LB_IX_E5, r32) >> 9);
  a3 = LB_IX_E3 + (ix_mulhi32(a3, r32) >> 9);
  int64_t a = LB_IX_E2 + (ix_mul64x32hi(r, a3) >> 10);      // r a3 in Q72
  a = LB_IX_E1 + (ix_mulhi(a, r) >> 9);
  const int64_t p = ix_mulhi(a, r);                         // Q71
  const int64_t t = (int64_t)LB_IX_LOAD(lb_ix_exp_t + (k & 511));   // 2^(j/512), Q62
  return t + (ix_mulhi(t, p) >> 7);                         // Q62, in [0.999, 2.002)
}

// e^y = 2^(k/512) (1 + p) for 2^-64 <= |y| <= 708, y given by its bits b
// (biased exponent E, sign neg): returns 2^(j/512) (1 + p) in Q62, in
// [0.999, 2.002), and k.
LB_IX_FN int64_t ix_exp_core(uint64_t b, int E, bool neg, int& kout) {
  // |y| in Q116 (exact: the 53-bit significand shifted left by E - 959 <= 73)
  const uint64_t M = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const int s = E - 959;
  uint64_t yhi, ylo;
  if (s >= 64) { yhi = M << (s - 64); ylo = 0; }
  else { yhi = s ? M >> (64 - s) : 0; ylo = M << s; }
  // k ~ rint(|y| 512 / ln2) from a single-precision copy of |y| (24 bits, truncated)
  const float yf = ix_float((uint32_t)((E - 1023 + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
  const uint32_t ak = ix_fbits(fmaf(yf, 738.65986f, 12582912.0f)) - 0x4B400000u;   // 1.5 2^23 shift
  // r = |y| - k ln2/512 in Q116, then Q73 (k < 2^20: 64 x 32-bit products)
  const uint64_t k0 = (uint64_t)ak * (LB_IX_L512_LO & 0xffffffffull);
  const uint64_t k1 = (uint64_t)ak * (LB_IX_L512_LO >> 32);
  const uint64_t klo = k0 + (k1 << 32);
  const uint64_t khi = (uint64_t)ak * LB_IX_L512_HI + (k1 >> 32) + (klo < k0 ? 1u : 0u);
  const uint64_t rlo = ylo - klo;
  const uint64_t rhi = yhi - khi - (ylo < klo ? 1u : 0u);
  int64_t r = (int64_t)((rhi << 21) | (rlo >> 43));
  int k = (int)ak;
  if (neg) { r = -r; k = -k; }
  kout = k;
  return ix_exp_finish(r, k);
}

LB_IX_FN double ix_exp(double y) {
  const uint64_t b = ix_bits(y);
  const int E = (int)((b >> 52) & 0x7ff);
  const bool neg = (b >> 63) != 0;
  if (E < 959) return 1.0;                                  // |y| < 2^-64 (and zeros, subnormals)
  if (((uint32_t)(b >> 32) & 0x7fffffffu) > 0x40862000u) return neg ? 0.0 : INFINITY;   // |y| > 708 (or NaN)
  int k;
  const int64_t res = ix_exp_core(b, E, neg, k);
  const int lz = ix_clz((uint64_t)res);                     // 1 or 2
  const uint64_t m53 = (((uint64_t)res << (lz - 1)) + (1ull << 9)) >> 10;   // [2^52, 2^53]
  const int biased = (k >> 9) + 1024 - lz;
  if (biased <= 0) return 0.0;
  return ix_double(((uint64_t)(biased - 1) << 52) + m53);
}

// e^y in unsigned Q58 fixed point (e^y 2^58, rounded to the nearest
// integer, ties up), for y < ln 2 (the result is below 2^59, so 32 of them
// add up without overflow); y <= -42 gives 0 (e^y < 2^-60).  Within 0.6 of
// the exact value, in units of 2^-58.  For sums of terms e^(L - max L):
// fixed-point terms add exactly on the integer pipes.
LB_IX_FN uint64_t ix_exp_q58(double y) {
  const uint64_t b = ix_bits(y);
  const int E = (int)((b >> 52) & 0x7ff);
  const bool neg = (b >> 63) != 0;
  if (E < 959) return 1ull << 58;                           // |y| < 2^-64
  if (neg && ((uint32_t)(b >> 32) & 0x7fffffffu) >= 0x40450000u) return 0;   // y <= -42
  int k;
  const int64_t res = ix_exp_core(b, E, neg, k);            // e^y = res 2^(k div 512 - 62)
  const int sh = 4 - (k >> 9);                              // to Q58; k div 512 <= 0 for y < ln 2
  if (sh >= 64) return 0;                                   // below 2^-59: rounds to 0
  return ((uint64_t)res + (1ull << (sh - 1))) >> sh;
}

LB_IX_FN double ix_log(double z) {
  const uint64_t b = ix_bits(z);
  const uint32_t hi = (uint32_t)(b >> 32);
  if (hi < 0x00100000u || hi >= 0x7ff00000u) return log(z);   // <= 0, subnormal, inf, NaN
  const int e = (int)(hi >> 20) - 1023;
  const uint64_t F = b & 0x000fffffffffffffull;
  const int j = (int)(F >> 43);
  const uint64_t M = F | 0x0010000000000000ull;
  // r = m C_j / 2^13 - 1 in Q65: the low 64 bits of M C_j (the product is 2^65 (1 + r))
  const int64_t r = (int64_t)(M * (uint64_t)LB_IX_LOAD(lb_ix_log_c + j));
  // log(1 + r) = r (1 - r (1/2 - r (1/3 - r (1/4 - r (1/5 - r/6))))).  The
  // steps for 1/5 and 1/4 enter the result times r^4 (|r| < 2^-9.8): 32-bit
  // precision (Q31, r in Q33) suffices there; 1/3, 1/2 and 1 in Q62.
  const int32_t r32 = (int32_t)(r >> 32);                   // Q33
  int32_t a4 = LB_IX_L5 - (ix_mulhi32(LB_IX_L6, r32) >> 1);
  a4 = LB_IX_L4 - (ix_mulhi32(a4, r32) >> 1);
  int64_t a = LB_IX_L3 - (ix_mul64x32hi(r, a4) >> 2);       // r a4 in Q64
  a = LB_IX_L2 - (ix_mulhi(a, r) >> 1);
  a = LB_IX_L1 - (ix_mulhi(a, r) >> 1);
  // p = a r as a full product (Q127), moved to Q116
  const int64_t phi = ix_mulhi(a, r);
  const uint64_t plo = (uint64_t)a * (uint64_t)r;
  uint64_t slo = (plo >> 11) | ((uint64_t)phi << 53);
  int64_t shi = phi >> 11;
  // + table entry -log(C_j / 2^13), Q116
  {
    const uint64_t tlo = LB_IX_LOAD(lb_ix_log_tlo + j);
    const int64_t thi = LB_IX_LOAD(lb_ix_log_thi + j);
    const uint64_t lo = slo + tlo;
    shi = shi + thi + (lo < slo ? 1 : 0);
    slo = lo;
  }
  // + e ln2, Q116
  if (e != 0) {
    const uint64_t ae = (uint64_t)(e < 0 ? -e : e);       // < 2^11: 64 x 32-bit products
    const uint64_t l0 = ae * (LB_IX_LN2_LO & 0xffffffffull);
    const uint64_t l1 = ae * (LB_IX_LN2_LO >> 32);
    uint64_t llo = l0 + (l1 << 32);
    uint64_t lhi = ae * LB_IX_LN2_HI + (l1 >> 32) + (llo < l0 ? 1u : 0u);
    if (e < 0) {
      llo = ~llo + 1;
      lhi = ~lhi + (llo == 0 ? 1 : 0);
    }
    const uint64_t lo = slo + llo;
    shi = (int64_t)((uint64_t)shi + lhi + (lo < slo ? 1 : 0));
    slo = lo;
  }
  // to double: sign, magnitude, normalise, round to 53 bits
  uint64_t sign = 0, mhi = (uint64_t)shi, mlo = slo;
  if (shi < 0) {
    sign = 0x8000000000000000ull;
    mlo = ~mlo + 1;
    mhi = ~mhi + (mlo == 0 ? 1 : 0);
  }
  if ((mhi | mlo) == 0) return 0.0;
  const int lz = mhi ? ix_clz(mhi) : 64 + ix_clz(mlo);
  uint64_t top;                                             // bits 127 - lz .. 64 - lz
  if (lz == 0) top = mhi;
  else if (lz < 64) top = (mhi << lz) | (mlo >> (64 - lz));
  else top = mlo << (lz - 64);
  const uint64_t m53 = (top >> 11) + ((top >> 10) & 1u);    // [2^52, 2^53] (no overflow at top ~ 2^64)
  const int biased = 11 - lz + 1023;                        // value = top 2^(11 - lz - 63)
  return ix_double(sign | (((uint64_t)(biased - 1) << 52) + m53));
}

// ---------------------------------------------------------------------------
// Fixed point for sums of terms e^(c + a log z - m): the K-integral nodes
// (lb_kint.cuh) keep each node's logarithm term in Q53 (an int64 holding
// value 2^53; |value| < 2^10), form it, its warp maximum and the shift by
// that maximum with integer instructions, and exponentiate the shifted
// term from Q53 straight into the Q58 sum.  No double is packed or unpacked
// between the steps, and no FP64 instruction runs.
// ---------------------------------------------------------------------------

// round(d 2^q) for |d| < 2^(62 - q), from the bit fields (ties away from 0;
// zero and subnormals give 0).
LB_IX_FN int64_t ix_fix(double d, int q) {
  const uint64_t b = ix_bits(d);
  const int E = (int)((b >> 52) & 0x7ff);
  const uint64_t M = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const int s = E - 1075 + q;                               // value 2^q = M 2^s
  int64_t m;
  if (E == 0 || s < -54) m = 0;
  else if (s >= 0) m = (int64_t)(M << s);
  else m = (int64_t)((M + (1ull << (-s - 1))) >> -s);
  return (b >> 63) ? -m : m;
}

// round(a b 2^-58): a in Q58 times b in Q53, in Q53 (|a b| below 2^10 in
// value); ties up.
LB_IX_FN int64_t ix_mul_q58(int64_t a, int64_t b) {
  const int64_t hi = ix_mulhi(a, b);
  const uint64_t lo = (uint64_t)a * (uint64_t)b;
  const uint64_t lo2 = lo + (1ull << 57);
  const uint64_t hi2 = (uint64_t)hi + (lo2 < lo ? 1u : 0u);
  return (int64_t)((hi2 << 6) | (lo2 >> 58));
}

// log z in Q53 for positive normal z (the reduction of ix_log; the sum
// -log(C_j / 2^13) + log(1 + r) in Q62 and e ln2 from its 94-bit form):
// within 0.56 units of 2^-53.  For this precision log(1 + r) stops at r^5
// (r^6/6 below 2^-61.4, and below 2^-56.6 in the first interval, j = 0,
// where r reaches 2^-9), and a step's error enters times r^k after k more
// steps, so 1/4 - r/5 and 1/3 - r(...) run in 32 bits (Q30), 1/2 - r(...)
// as a 64 x 32-bit product and only the last two in 64 bits.  With r in
// Q64 every product lands in its sum's format without a shift.
// Zero, negative, subnormal, infinite and NaN z give -2^62 (a term that
// vanishes); the callers pass positive normal z.
LB_IX_FN int64_t ix_log_q53(double z) {
  const uint64_t b = ix_bits(z);
  const uint32_t hi = (uint32_t)(b >> 32);
  if (hi < 0x00100000u || hi >= 0x7ff00000u) return -(1ll << 62);
  const int e = (int)(hi >> 20) - 1023;
  const uint64_t F = b & 0x000fffffffffffffull;
  const int j = (int)(F >> 43);
  // r = m C_j / 2^13 - 1: the low 64 bits of M C_j are 2^65 r; r in Q64
  const int64_t r = (int64_t)((F | 0x0010000000000000ull) * (uint64_t)LB_IX_LOAD(lb_ix_log_c + j)) >> 1;
  const int32_t r32 = (int32_t)(r >> 32);                   // Q32
  int32_t a3 = LB_IX_LQ4 - ix_mulhi32(LB_IX_LQ5, r32);      // Q30
  a3 = LB_IX_LQ3 - ix_mulhi32(a3, r32);
  int64_t a = LB_IX_L2 - ix_mul64x32hi(r, a3);              // Q62
  a = LB_IX_L1 - ix_mulhi(a, r);
  // log(1 + r) = a r plus -log(C_j / 2^13), Q62: |f| < 0.7
  const int64_t f = ix_mulhi(a, r) + (int64_t)LB_IX_LOAD(lb_ix_log_t62 + j);
  // e ln2 = e (A 2^-30 + B 2^-62 + C 2^-94): the last two parts with f in Q62
  const int64_t lo62 = (int64_t)e * LB_IX_LN2Q_B + (((int64_t)e * LB_IX_LN2Q_C) >> 32) + f;
  return (int64_t)((uint64_t)((int64_t)e * LB_IX_LN2Q_A) << 23) + ((lo62 + (1ll << 8)) >> 9);
}

// e^(d 2^-53) in unsigned Q58 (as ix_exp_q58) for d <= 0 in Q53; d <= -42
// (in value) gives 0.  The reduction r = |y| - k ln2/512 is formed in Q64
// modulo 2^64 (exact, as |r| < 2^-10.2) and carried to Q73.
LB_IX_FN uint64_t ix_exp_q58_fx(int64_t d) {
  if (d <= -(42ll << 53)) return 0;
  const uint64_t ad = (uint64_t)(-d);                       // |y| in Q53, below 2^58.4
  // k ~ rint(|y| 512 / ln2) from a single-precision copy of |y| (in Q21)
  const float yf = (float)(int32_t)(ad >> 32);
  const uint32_t ak = ix_fbits(fmaf(yf, 738.65986f / 2097152.0f, 12582912.0f)) - 0x4B400000u;
  // y = -|y| = -k ln2/512 + r: r = k ln2/512 - |y|, in Q64 modulo 2^64, then Q73
  const uint64_t r64 = (uint64_t)ak * LB_IX_L512_H + (((uint64_t)ak * LB_IX_L512_M) >> 32) - (ad << 11);
  const int64_t r = (int64_t)(r64 << 9);
  const int k = -(int)ak;
  const int64_t res = ix_exp_finish(r, k);                  // e^y = res 2^(k div 512 - 62)
  const int sh = 4 - (k >> 9);                              // k div 512 <= 0
  if (sh >= 64) return 0;
  return ((uint64_t)res + (1ull << (sh - 1))) >> sh;
}

// Shared reduction of ix_rcp and ix_rsqrt: z = 2^e m, m in [1, 2),
// j = the top 9 fraction bits, r = m C_j / 2^13 - 1 (exact, |r| < 2^-9.8)
// returned as 2^65 r (the low 64 bits of M C_j, as in ix_log), and C_j.
LB_IX_FN int64_t ix_reduce_cj(uint64_t b, int& e, int& j, uint64_t& cj) {
  e = (int)(b >> 52) - 1023;
  const uint64_t F = b & 0x000fffffffffffffull;
  j = (int)(F >> 43);
  cj = (uint64_t)LB_IX_LOAD(lb_ix_log_c + j);
  return (int64_t)((F | 0x0010000000000000ull) * cj);
}

// Double from W in [2^61, 2^63) (value W 2^-62, rounded to 53 bits) times 2^-h.
LB_IX_FN double ix_pack(uint64_t W, int h) {
  const int lz = ix_clz(W);                                 // 1 or 2
  const uint64_t m53 = ((W << (lz - 1)) + (1ull << 9)) >> 10;   // [2^52, 2^53]
  return ix_double(((uint64_t)(1023 - lz - h) << 52) + m53);
}

// 1/z for positive normal z below 2^1022 (others: the division 1/z):
// 1/m = (C_j / 2^13) / (1 + r) with 1/(1 + r) = sum_{k<=6} (-r)^k (|r|^7 <
// 2^-68); the inner three steps in Q30 (32-bit multiplies), the outer in
// Q62.  Error below 0.51 ulp (checked on the CPU against exact rationals).
LB_IX_FN double ix_rcp(double z) {
  const uint64_t b = ix_bits(z);
  const uint32_t hi = (uint32_t)(b >> 32);
  if (hi < 0x00100000u || hi >= 0x7fd00000u) return 1.0 / z;
  int e, j;
  uint64_t cj;
  const int64_t r = ix_reduce_cj(b, e, j, cj);              // Q65
  const int32_t r32 = (int32_t)(r >> 32);                   // Q33
  int32_t a = (1 << 30) - (ix_mulhi32(1 << 30, r32) >> 1);  // Q30: 1 - r
  a = (1 << 30) - (ix_mulhi32(a, r32) >> 1);
  a = (1 << 30) - (ix_mulhi32(a, r32) >> 1);
  int64_t p = (1ll << 62) - (ix_mul64x32hi(r, a) >> 1);     // Q62 (r a in Q63)
  p = (1ll << 62) - (ix_mulhi(r, p) >> 1);
  p = (1ll << 62) - (ix_mulhi(r, p) >> 1);                  // 1/(1 + r), Q62
  // (C_j / 2^13) p in Q62: (2 p) (C_j 2^50) / 2^64
  const uint64_t W = ix_umulhi((uint64_t)p << 1, cj << 50);
  return ix_pack(W, e);
}

// 1/sqrt(z) for positive normal z (others: the libm 1/sqrt): z = 2^(2h+o) m
// (o = 0 or 1), m^-1/2 = sqrt(C_j / 2^13) (1 + r)^-1/2 with the binomial
// series to r^6 (|r|^7 < 2^-68), times 2^-1/2 for odd exponents.  Error
// below 0.52 ulp (checked on the CPU).
LB_IX_FN double ix_rsqrt(double z) {
  const uint64_t b = ix_bits(z);
  const uint32_t hi = (uint32_t)(b >> 32);
  if (hi < 0x00100000u || hi >= 0x7ff00000u) return 1.0 / sqrt(z);
  int e, j;
  uint64_t cj;
  const int64_t r = ix_reduce_cj(b, e, j, cj);              // Q65
  const int32_t r32 = (int32_t)(r >> 32);                   // Q33
  int32_t a = LB_IX_R5 - (ix_mulhi32(LB_IX_R6, r32) >> 1);  // Q30
  a = LB_IX_R4 - (ix_mulhi32(a, r32) >> 1);
  a = LB_IX_R3 - (ix_mulhi32(a, r32) >> 1);
  int64_t p = LB_IX_R2 - (ix_mul64x32hi(r, a) >> 1);        // Q62
  p = LB_IX_R1 - (ix_mulhi(r, p) >> 1);
  p = (1ll << 62) - (ix_mulhi(r, p) >> 1);                  // (1 + r)^-1/2, Q62
  uint64_t W = ix_umulhi((uint64_t)LB_IX_LOAD(lb_ix_rsq_t + j), (uint64_t)p << 1);   // Q62
  if (e & 1) W = ix_umulhi(W, LB_IX_RSQRT_HALF);
  return ix_pack(W, e >> 1);                                // e >> 1 = floor(e / 2)
}

#if defined(__CUDACC__)
// ix_log as a called function, for the per-pair call sites of large kernels:
// one copy of its code instead of one per call site keeps the tile kernel's
// hot code within the instruction cache (measured 2.5 % faster).
static __device__ __noinline__ double ix_log_call(double z) { return ix_log(z); }
static __device__ __noinline__ double ix_rcp_call(double z) { return ix_rcp(z); }
static __device__ __noinline__ double ix_rsqrt_call(double z) { return ix_rsqrt(z); }
#endif

}  // namespace lb
