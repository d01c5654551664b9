// lb_expr32.cuh -- FP32-mixed form of the expressions (device code).
//
// Same expressions and dispatch as lb_expr.cuh / lb_kint.cuh, evaluated in
// single precision on the FP32 pipe, which on GB300 issues 62 times faster
// than FP64.  Inputs and outputs are float.  The error target is 2e-6 of the
// error scale max(|f|, 1, |x df/dx|, |v df/dv|): every intermediate of these
// expressions is within a few tens of units in the last place of that scale,
// so single precision suffices throughout.
#pragma once

#include "lb_expr.cuh"
#include "kquad_tables.h"

namespace lb {

// Domain edges (same convention as special_value), in float.
template <int KIND>
__device__ __forceinline__ bool special_value32(float v, float x, float* r) {
  if (KIND == KIND_I) {
    if (isnan(v) || isnan(x) || v < 0.0f || x < 0.0f || (isinf(v) && isinf(x))) { *r = __int_as_float(0x7fc00000); return true; }
    if (isinf(x)) { *r = INFINITY; return true; }
    if (isinf(v)) { *r = -INFINITY; return true; }
    if (x == 0.0f) { *r = (v == 0.0f) ? 0.0f : -INFINITY; return true; }
  } else {
    if (isnan(v) || isnan(x) || x < 0.0f || (isinf(v) && isinf(x))) { *r = __int_as_float(0x7fc00000); return true; }
    if (isinf(x)) { *r = -INFINITY; return true; }
    if (x == 0.0f || isinf(v)) { *r = INFINITY; return true; }
  }
  return false;
}

// Region dispatch in float (FP64 compares would cost more than the FP32
// evaluation itself).  A pair within one float rounding of a threshold may
// land on the other side than in the FP64 path; both expressions are
// accurate there.
__device__ __forceinline__ int classify32(float v, float x, int mode) {
  if (mode == MODE_TIGHT) {
    if ((x > 30.0f && v < 13.6f) || (x > 59.6925f && v * v < 3.24f * x)) return R_MU20;
    if (v > 230.0f) return R_U4;
    if (v > 70.0f) return R_U6;
    if (v > 28.0f) return R_U9;
    if ((x > 25.0f && v > 0.7f) || v > 16.0f) return R_U13;
    return R_FALLBACK;
  }
  const float lx = logf(x), lv = logf(v);
  const bool mu20 = (x > 30.0f && v < 15.3919f) || ((0.5113f * lx + 0.7939f > lv) && x > 59.6925f);
  const bool u13 = (x > 19.6931f && v > 0.7f) || v > 12.6964f;
  if (mode == MODE_PAPER_CPU) {
    if ((x > 1400.0f && v < 3.05f) || ((0.6229f * lx - 3.2318f > lv) && v > 3.1f)) return R_MU3;
    if (mu20) return R_MU20;
    if ((x > 274.2377f && v > 0.3f) || v > 163.6993f) return R_U4;
    if ((x > 84.4153f && v > 0.46f) || v > 56.9971f) return R_U6;
    if ((x > 35.9074f && v > 0.6f) || v > 20.1534f) return R_U9;
    if (u13) return R_U13;
    return R_FALLBACK;
  }
  if (mu20) return R_MU20;
  if (u13) return R_U13;
  return R_FALLBACK;
}

template <int KIND, int K>
__device__ __forceinline__ float mu_expr32(float v, float x) {
  const float mu = 4.0f * v * v;
  const float inv8x = 1.0f / (8.0f * x);
  float P = 1.0f;
#pragma unroll
  for (int k = K; k >= 1; --k) {
    const float odd = (float)((2 * k - 1) * (2 * k - 1));
    float r = (mu - odd) * (inv8x * (1.0f / (float)k));
    if (KIND == KIND_I) r = -r;
    P = fmaf(r, P, 1.0f);
  }
  const float S = fabsf(P);
  if (KIND == KIND_I) return x + logf(S * rsqrtf((float)kTwoPi * x));
  return logf(S * sqrtf((float)kPi / (2.0f * x))) - x;
}

template <int KIND, int K>
__device__ __forceinline__ float u_expr32(float v, float x) {
  const float xp = x / v;
  const float r = (xp < 1e18f) ? sqrtf(fmaf(xp, xp, 1.0f)) : xp;
  const float t = 1.0f / r;
  const float p = t * t;
  float q = t / v;
  if (KIND == KIND_K) q = -q;
  float acc = debye_P<float>(K, p);
#pragma unroll
  for (int k = K - 1; k >= 1; --k) acc = fmaf(acc, q, debye_P<float>(k, p));
  const float S = fabsf(fmaf(acc, q, 1.0f));
  const float eta = r + logf(xp / (1.0f + r));
  if (KIND == KIND_I) return fmaf(v, eta, logf(S * rsqrtf((float)kTwoPi * v * r)));
  return fmaf(-v, eta, logf(S * sqrtf((float)kPi / (2.0f * v * r))));
}

// Power series of I_v in single precision.
__device__ __forceinline__ float series_log_i32(float v, float x) {
  const float y = 0.25f * x * x;
  const float kpk = 0.5f * (sqrtf(fmaf(x, x, v * v)) - v);
  float term = 1.0f, T = 0.0f;
  float k = 1.0f;
  for (int it = 0; it < 400; ++it) {
    term *= y / (k * (k + v));
    T += term;
    if (k > kpk && term <= 1.5e-8f * (1.0f + T)) break;
    k += 1.0f;
  }
  float res = log1pf(T) - lgammaf(v + 1.0f);
  if (v != 0.0f) res = fmaf(v, logf(0.5f * x), res);
  return res;
}

// K integral, Gauss rules of lb_kint.cuh evaluated in single precision
// (float copies of the tables).  Warp-cooperative; all lanes pass the same pair.
__device__ __forceinline__ float kint_gauss32(float v, float x, int lane) {
  const float beta = 16.0f / (2.0f * v + 1.0f);
  const float logbeta = logf(beta);
  const float vm = v - 0.5f, tx = 2.0f * x;
  const float* gu;
  const float* gw;
  int ng;
  if (v >= 0.9f || x >= 0.25f) { gu = lb_kqf_g32_logu; gw = lb_kqf_g32_logw; ng = 32; }
  else if (v >= 0.4f || x >= 1e-3f) { gu = lb_kqf_g64_logu; gw = lb_kqf_g64_logw; ng = 64; }
  else { gu = lb_kqf_g128_logu; gw = lb_kqf_g128_logw; ng = 128; }
  const float *hs, *hy, *hc;
  int nh;
  if (v <= 1.2f) { hs = lb_kqf_hl32_s; hy = lb_kqf_hl32_y; hc = lb_kqf_hl32_c; nh = 32; }
  else if (v <= 5.0f) { hs = lb_kqf_hl48_s; hy = lb_kqf_hl48_y; hc = lb_kqf_hl48_c; nh = 48; }
  else { hs = lb_kqf_hq32_s; hy = lb_kqf_hq32_y; hc = lb_kqf_hq32_c; nh = 32; }
  float L[6];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = lane + 32 * k;
    L[k] = -INFINITY;
    if (32 * k < ng) {
      const float logu = __ldg(gu + j);
      const float ub = expf(beta * logu);
      L[k] = __ldg(gw + j) + logbeta - ub + fmaf(vm, logf(tx + ub), 7.0f * logu);
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = lane + 32 * k;
    L[4 + k] = -INFINITY;
    if (j < nh) {
      const float sj = __ldg(hs + j);
      L[4 + k] = fmaf(vm, __ldg(hy + j) + logf(sj + tx), __ldg(hc + j));
    }
  }
  float m = L[0];
#pragma unroll
  for (int i = 1; i < 6; ++i) m = fmaxf(m, L[i]);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const bool live = (k < 4) ? (32 * k < ng) : (32 * (k - 4) < nh && L[k] > -INFINITY);
    if (live) s += expf(L[k] - m);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return m + logf(s);
}

// log-prefactor of the K integral: log(sqrt(pi) e^{-x} / (Gamma(v+1/2) (2x)^v))
__device__ __forceinline__ float kint_prefactor32(float v, float x) {
  return (float)kHalfLogPi - lgammaf(v + 0.5f) - fmaf(v, logf(2.0f * x), x);
}

}  // namespace lb
