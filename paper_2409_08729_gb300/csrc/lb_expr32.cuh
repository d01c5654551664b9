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
// w: WIDE_I / WIDE_K for values of log I / log K, which take the wider
// mu_20 and U_13 ranges of the FP64 form (tight_mu20_w, tight_u13_w; there
// the truncation error is below 3.1e-16; in single precision the mu_20
// terms grow to at most 3 there, and the Debye sums' rounding, bounded by
// 6e-8 sum_k sum_i |c_ki| / v^k, stays below 5e-8 for v > 10).
__device__ __forceinline__ int classify32(float v, float x, int mode, int w = WIDE_NONE) {
  if (mode == MODE_TIGHT) {
    bool mu = (x > 30.0f && v < 13.6f) || (x > 59.6925f && v * v < 3.24f * x);
    if (w == WIDE_K) mu = mu || (x > 18.5f && v < 9.5f) || (x > 20.0f && v < 12.5f) || (x > 22.0f && v < 13.6f);
    if (w == WIDE_I) mu = mu || (x > 19.0f && v < 4.5f) || (x > 21.0f && v < 7.5f) || (x > 23.0f && v < 9.5f);
    if (mu) return R_MU20;
    if (v > 230.0f) return R_U4;
    if (v > 70.0f) return R_U6;
    if (v > 28.0f) return R_U9;
    bool u = (x > 25.0f && v > 0.7f) || v > 16.0f;
    if (w == WIDE_K) u = u || (x > 19.0f && v > 10.0f) || (x > 14.0f && v > 14.0f);
    if (w == WIDE_I) u = u || (x > 19.5f && v > 10.0f) || (x > 17.5f && v > 12.0f) || (x > 14.5f && v > 14.0f);
    if (u) return R_U13;
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
  const float inv_v = 1.0f / v;
  const float xp = x * inv_v;
  float r, t;
  if (xp < 1e18f) {
    const float r2 = fmaf(xp, xp, 1.0f);
    t = rsqrtf(r2);                                  // single-precision estimate (2 ulp)
    r = r2 * t;
  } else {
    r = xp;
    t = 1.0f / xp;
  }
  const float p = t * t;
  float q = t * inv_v;
  if (KIND == KIND_K) q = -q;
  float acc = debye_P<float>(K, p);
#pragma unroll
  for (int k = K - 1; k >= 1; --k) acc = fmaf(acc, q, debye_P<float>(k, p));
  const float S = fabsf(fmaf(acc, q, 1.0f));
  const float eta = r + logf(__fdividef(xp, 1.0f + r));
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
    term *= __fdividef(y, k * (k + v));             // 2 ulp per ratio: within the path's budget
    T += term;
    if (k > kpk && term <= 1.5e-8f * (1.0f + T)) break;
    k += 1.0f;
  }
  float res = log1pf(T) - lgammaf(v + 1.0f);
  if (v != 0.0f) res = fmaf(v, logf(0.5f * x), res);
  return res;
}

// K integral, Gauss rules of lb_kint.cuh evaluated in single precision
// (float copies of the tables): the one-slot rules for 2 <= v <= 16.5, the
// packed rule for 1.2 < v <= 5 below that, the fixed rules, and the split g
// rule for v < 0.4, x < 1e-3 (see kint_sums_split: the nodes anchored at
// s1 = 128 x carry their terms less C = 2 v log s1 and are shifted by
// m - C).  Warp-cooperative; all lanes pass the same pair.
// One order for every pair of a call: u_j^beta of the three u rules and the
// one-slot rule's s0 u_j^beta once per block (as KintScalar; same operations,
// same results).
struct KintScalar32 {
  float ub24[24], ub32[32], ub64[64];
  float sg[22];                                    // s0 u_j^beta of the one-slot rule of v (if any)
};

__device__ __forceinline__ void kint_scalar_setup32(KintScalar32& ks, float v) {
  const int tid = threadIdx.x;
  const float beta = 16.0f / (2.0f * v + 1.0f);
  if (tid < 24) ks.ub24[tid] = expf(beta * __ldg(lb_kqf_g24_logu + tid));
  else if (tid < 56) ks.ub32[tid - 24] = expf(beta * __ldg(lb_kqf_g32_logu + tid - 24));
  else if (tid < 120) ks.ub64[tid - 56] = expf(beta * __ldg(lb_kqf_g64_logu + tid - 56));
  else if (tid >= 128 && tid < 150 && v >= 2.0f && v <= 16.5f) {
    const int j = tid - 128;
    if (v < 7.0f) ks.sg[j] = expf(fmaf(beta, __ldg(lb_kqf_g22_logu + j), (float)LB_KQ_LOG8));
    else if (j < 12) ks.sg[j] = expf(fmaf(beta, __ldg(lb_kqf_g12_logu + j), (float)LB_KQ_LOG3));
  }
  __syncthreads();
}

// The summand exps (arguments <= 0, the largest terms near 0) use the fast
// single-precision exp: about 2e-7 relative error near 0, growing like
// 6e-8 |argument| on terms that weigh e^-|argument|, so the sum moves by
// about 2e-7 relative, well inside the FP32 path's 2e-6.
// Warp maximum of a float through an order-preserving integer key (one
// integer reduction instead of five shuffle rounds).
__device__ __forceinline__ float warp_max32(float a) {
  const int k = __float_as_int(a);
  const int key = __reduce_max_sync(0xffffffffu, k >= 0 ? k : (k ^ 0x7fffffff));
  return __int_as_float(key >= 0 ? key : (key ^ 0x7fffffff));
}

// beta = 16/(2v + 1) and log beta are per pair: the caller computes them
// once per lane and passes the shuffled values.
__device__ __forceinline__ float kint_gauss32(float v, float x, float beta, float logbeta, int lane,
                                              const KintScalar32* ks = nullptr) {
  const float vm = v - 0.5f, vp = v + 0.5f, tx = 2.0f * x;
  if (v >= 2.0f && v <= 16.5f) {
    // the one-slot rules of the FP64 path (kint_sum_one): int_0^inf F split at
    // s0 = 8 (22 g + 10 h nodes, v < 7) or s0 = 3 (12 + 20), [0, s0] with
    // s = s0 u^beta, [s0, inf) by Gauss-Laguerre in s - s0: one lane slot
    // instead of two
    const bool r4 = v < 7.0f;
    const int ng = r4 ? 22 : 12;
    const float ls0 = r4 ? (float)LB_KQ_LOG8 : (float)LB_KQ_LOG3;
    const bool isg = lane < ng;
    float s, y, c;
    if (isg) {
      s = ks ? ks->sg[lane] : expf(fmaf(beta, __ldg((r4 ? lb_kqf_g22_logu : lb_kqf_g12_logu) + lane), ls0));
      y = 0.0f;
      c = __ldg((r4 ? lb_kqf_g22_c : lb_kqf_g12_c) + lane) + fmaf(vp, ls0, logbeta);
    } else {
      const int j = lane - ng;
      s = __ldg((r4 ? lb_kqf_hq10o8_s : lb_kqf_hq20o3_s) + j);
      y = __ldg((r4 ? lb_kqf_hq10o8_y : lb_kqf_hq20o3_y) + j);
      c = __ldg((r4 ? lb_kqf_hq10o8_c : lb_kqf_hq20o3_c) + j);
    }
    const float L = fmaf(vm, logf(tx + s) + y, c) - (isg ? s : 0.0f);
    const float m = warp_max32(L);
    float sum = __expf(L - m);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    return m + logf(sum);
  }
  if (v > 1.2f && v <= 5.0f) {
    // 24 g + 40 h nodes in two lane slots (as kint_sumq_g24h40)
    const bool isg = lane < 24;
    const int jh = isg ? 0 : lane - 24;
    const float s = isg ? (ks ? ks->ub24[lane] : expf(beta * __ldg(lb_kqf_g24_logu + lane))) : __ldg(lb_kqf_hl40_s + jh);
    const float y0 = isg ? 0.0f : __ldg(lb_kqf_hl40_y + jh);
    const float c0 = isg ? __ldg(lb_kqf_g24_c + lane) + logbeta : __ldg(lb_kqf_hl40_c + jh);
    const float L0 = fmaf(vm, logf(tx + s) + y0, c0) - (isg ? s : 0.0f);
    const float sh = __ldg(lb_kqf_hl40_s + 8 + lane);
    const float L1 = fmaf(vm, __ldg(lb_kqf_hl40_y + 8 + lane) + logf(sh + tx), __ldg(lb_kqf_hl40_c + 8 + lane));
    const float m = warp_max32(fmaxf(L0, L1));
    float sum = __expf(L0 - m) + __expf(L1 - m);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    return m + logf(sum);
  }
  const int ng = (v >= 0.9f || x >= 0.25f) ? 32 : ((v >= 0.4f || x >= 1e-3f) ? 64 : 0);
  const float *hs, *hy, *hc;
  int nh;
  if (v <= 1.2f) { hs = lb_kqf_hl32_s; hy = lb_kqf_hl32_y; hc = lb_kqf_hl32_c; nh = 32; }
  else if (v <= 5.0f) { hs = lb_kqf_hl48_s; hy = lb_kqf_hl48_y; hc = lb_kqf_hl48_c; nh = 48; }
  else { hs = lb_kqf_hq32_s; hy = lb_kqf_hq32_y; hc = lb_kqf_hq32_c; nh = 32; }
  float L[7];
  bool live[7], rel[7];
  const float sx = 128.0f * x;
  const float y1 = (ng == 0) ? logf(sx) : 0.0f;     // log s1
  const float C = 2.0f * v * y1;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    L[k] = -INFINITY;
    live[k] = false;
    rel[k] = false;
    if (ng != 0) {
      if (k < 2 && 32 * k < ng) {
        const int j = lane + 32 * k;
        const float logu = ng == 32 ? __ldg(lb_kqf_g32_logu + j) : __ldg(lb_kqf_g64_logu + j);
        const float c = ng == 32 ? __ldg(lb_kqf_g32_c + j) : __ldg(lb_kqf_g64_c + j);
        const float ub = ks ? (ng == 32 ? ks->ub32[j] : ks->ub64[j]) : expf(beta * logu);
        L[k] = c + logbeta - ub + vm * logf(tx + ub);
        live[k] = true;
      }
    } else if (k < 2) {                               // [0, s1]: s = s1 r, r = u^beta
      const int j = lane + 32 * k;
      const float r = ks ? ks->ub64[j] : expf(beta * __ldg(lb_kqf_g64_logu + j));
      L[k] = fmaf(vm, logf(r + 0.015625f), __ldg(lb_kqf_g64_c + j) + logbeta) - sx * r;
      live[k] = true;
      rel[k] = true;
    } else {                                          // [s1, 1] in y = log s, panels as in FP64
      float a, b, t, lw;
      bool anchored;
      if (k == 2) {
        const int j = lane & 15;
        t = __ldg(lb_kqf_gl16_t + j);
        lw = __ldg(lb_kqf_gl16_logw + j);
        anchored = lane < 16;
        if (anchored) { a = 0.0f; b = fminf(8.0f, -4.0f - y1); }
        else { a = fmaxf(y1, -4.0f); b = 0.0f; }
      } else {
        t = __ldg(lb_kqf_gl32_t + lane);
        lw = __ldg(lb_kqf_gl32_logw + lane);
        anchored = k == 3;
        if (anchored) { a = 8.0f; b = fminf(40.0f, -4.0f - y1); }
        else { a = fmaxf(y1 + 40.0f, -40.0f); b = -4.0f; }
      }
      if (b > a) {
        const float o = fmaf(b - a, t, a);
        const float lwb = lw + logf(b - a);
        if (anchored) {
          const float eo = expf(o);
          L[k] = fmaf(vm, logf(eo + 0.015625f), fmaf(vp, o, lwb)) - sx * eo;
        } else {
          const float sv = expf(o);
          L[k] = fmaf(vm, logf(sv + tx), fmaf(vp, o, lwb)) - sv;
        }
        live[k] = true;
        rel[k] = anchored;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = lane + 32 * k;
    L[5 + k] = -INFINITY;
    live[5 + k] = j < nh;
    rel[5 + k] = false;
    if (j < nh) {
      const float sj = __ldg(hs + j);
      L[5 + k] = fmaf(vm, __ldg(hy + j) + logf(sj + tx), __ldg(hc + j));
    }
  }
  // closed-form flat middle of the split rule (int e^{2 v y} dy over
  // [y1 + 40, -40], w = -80 - y1), less C
  float Lflat = -INFINITY;
  const float w = -80.0f - y1;
  if (ng == 0 && w > 0.0f) Lflat = (v == 0.0f) ? logf(w) : fmaf(80.0f, v, logf(expm1f(2.0f * v * w) / (2.0f * v)));
  float m = Lflat + C;
#pragma unroll
  for (int i = 0; i < 7; ++i) m = fmaxf(m, rel[i] ? L[i] + C : L[i]);
  m = warp_max32(m);
  const float mr = m - C;
  float s = (lane == 0 && Lflat > -INFINITY) ? __expf(Lflat - mr) : 0.0f;
#pragma unroll
  for (int k = 0; k < 7; ++k)
    if (live[k]) s += __expf(L[k] - (rel[k] ? mr : m));
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return m + logf(s);
}

// log-prefactor of the K integral: log(sqrt(pi) e^{-x} / (Gamma(v+1/2) (2x)^v))
__device__ __forceinline__ float kint_prefactor32(float v, float x) {
  return (float)kHalfLogPi - lgammaf(v + 0.5f) - fmaf(v, logf(2.0f * x), x);
}

}  // namespace lb
