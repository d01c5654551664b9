// lb_df.cuh -- double-float arithmetic: a value held as an unevaluated sum
// h + l of two single-precision numbers (|l| <= ulp(h)), about 48
// significant bits.
//
// On GB300 the FP64 pipe retires 2 operations per SM per clock and the FP32
// pipe 128, so one FP64 instruction costs as much pipe time as about 64
// FP32 instructions.  Parts of a sum whose share of the result is small
// (below 1e-3 of it) need no more than double-float accuracy: its relative
// error of a few 2^-48 on such a part is below 1e-17 of the result.  The
// expressions (lb_expr.cuh) evaluate those parts -- the high-order terms of
// their Horner sums -- with these operations, which cost 7 to 15 FP32
// instructions each, and the leading terms in FP64.
//
// The operations are the error-free transformations of T. J. Dekker ("A
// floating-point technique for extending the available precision", Numer.
// Math. 18, 1971) and D. E. Knuth (TAOCP vol. 2, two-sum), with the product
// error taken by a fused multiply-add.  Conversions from and to double run
// on the integer pipe (bit fields), not through FP64 conversion
// instructions.  The functions also compile for the host (without
// __CUDACC__), with the same results where the host has fmaf and IEEE
// single precision, for the CPU tests.
#pragma once

#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define LB_DF_FN __host__ __device__ __forceinline__
#else
#include <string.h>
#define LB_DF_FN static inline
#endif

namespace lb {

struct dfloat {
  float h, l;
};

LB_DF_FN uint32_t df_fbits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
LB_DF_FN float df_bitsf(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
LB_DF_FN uint64_t df_dbits(double d) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
#endif
}
LB_DF_FN double df_bitsd(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
LB_DF_FN float df_fma(float a, float b, float c) { return fmaf(a, b, c); }

// d as a double-float: h = d cut to 24 significant bits, l = the other 29
// bits rounded to a float.  |d| below 2^-126 gives 0; l is dropped (0) for
// |d| below 2^-74.  The callers' values are below 2^100 in magnitude.
LB_DF_FN dfloat df_from_double(double d) {
  const uint64_t b = df_dbits(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sgn = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
  dfloat r;
  if (e < -126) {
    r.h = 0.0f;
    r.l = 0.0f;
    return r;
  }
  r.h = df_bitsf(sgn | ((uint32_t)(e + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  if (e < -74) {
    r.l = 0.0f;
    return r;
  }
  // the low 29 fraction bits, worth 2^(e - 52) each (exact in the product:
  // a float times a power of two in range)
  const float rest = (float)(lo & 0x1fffffffu) * df_bitsf((uint32_t)(e - 52 + 127) << 23);
  r.l = df_bitsf(df_fbits(rest) | sgn);
  return r;
}

// A float as a double, from its bit fields (zero and subnormals give zero).
LB_DF_FN double df_f2d(float f) {
  const uint32_t u = df_fbits(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint64_t s = (uint64_t)(u & 0x80000000u) << 32;
  if (ex == 0) return df_bitsd(s);
  return df_bitsd(s | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

// h + l rounded to double: one FP64 addition (exact for a normalized pair
// within the double's 53 bits).
LB_DF_FN double df_to_double(dfloat a) { return df_f2d(a.h) + df_f2d(a.l); }

LB_DF_FN dfloat df_make(float h, float l) {
  dfloat r;
  r.h = h;
  r.l = l;
  return r;
}

// a * t + c (Horner step): the product's error by an FMA, the sum by
// Knuth's two-sum, then renormalized.  15 FP32 instructions.
LB_DF_FN dfloat df_mul_add(dfloat a, dfloat t, dfloat c) {
  const float p = a.h * t.h;
  float e = df_fma(a.h, t.h, -p);
  e = df_fma(a.h, t.l, e);
  e = df_fma(a.l, t.h, e);
  const float s = p + c.h;
  const float bp = s - p;
  const float e2 = (p - (s - bp)) + (c.h - bp);
  e = (e + e2) + c.l;
  dfloat r;
  r.h = s + e;
  r.l = e - (r.h - s);
  return r;
}

// a * b.  7 FP32 instructions.
LB_DF_FN dfloat df_mul(dfloat a, dfloat b) {
  const float p = a.h * b.h;
  float e = df_fma(a.h, b.h, -p);
  e = df_fma(a.h, b.l, e);
  e = df_fma(a.l, b.h, e);
  dfloat r;
  r.h = p + e;
  r.l = e - (r.h - p);
  return r;
}

// a + b.  11 FP32 instructions.
LB_DF_FN dfloat df_add(dfloat a, dfloat b) {
  const float s = a.h + b.h;
  const float bp = s - a.h;
  float e = (a.h - (s - bp)) + (b.h - bp);
  e = e + (a.l + b.l);
  dfloat r;
  r.h = s + e;
  r.l = e - (r.h - s);
  return r;
}

}  // namespace lb
