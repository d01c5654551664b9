// lb_kint.cuh -- warp-cooperative evaluation of the K integral (device code).
//
// Paper Sec. 3.2, Eq. "log Kv integral" (Rothwell's representation):
//   log K_v(x) = log(pi)/2 - lgamma(v + 1/2) - v log(2x) - x
//              + log int_0^1 [g(u) + h(u)] du,
//   g(u) = beta exp(-u^beta) (2x + u^beta)^(v-1/2) u^(n-1),  beta = 2n/(2v+1), n = 8,
//   h(u) = exp(-1/u) u^(-2v-1) (2xu + 1)^(v-1/2).
// With s = u^beta in g and s = 1/u in h both pieces are pieces of one
// integral, int_0^1 and int_1^inf of F(s) = e^{-s} (s (s + 2x))^(v-1/2) ds.
//
// One warp evaluates one pair: its lanes split the quadrature nodes, each lane
// keeps the logarithms of its weighted terms in registers, and two warp
// shuffles reductions form log sum exp (Eq. "log sum trick") with the exact
// maximum as shift.
//
// Rules:
//   LB_TIGHT: Gauss rules (tables in kquad_tables.h).  g: Gauss-Legendre in u
//     with 32 nodes (v >= 0.9 or x >= 0.25), 64 (v >= 0.4 or x >= 1e-3) or 128;
//     small x with v away from 1/2 needs more, because (2x + u^beta)^(v-1/2)
//     turns sharply near u = (2x)^(1/beta).  h: Gauss-Legendre in log s on
//     [1, 100] (32 nodes for v <= 1.2, 48 for v <= 5) or Gauss-Laguerre in
//     s - 1 (32 nodes, v > 5).  Node counts were chosen so the rule error
//     stays below 1e-16 over v in [0, 16], x in [1e-6, 30] (the fallback
//     region of the tight dispatch).
//   LB_PAPER_GPU: composite Simpson on u in [0, 1], N = 600 (paper Sec. 3.2)
//     with weights 4 (odd k), 2 (even k), 1 (k = N), the constant read as
//     1/(3N), f(0) = 0, and the paper's heuristic maxima log g(1) and
//     log h(u*), u* = 1/2 (v < 2) or 1/(2v), as log-sum-exp shifts.
#pragma once

#include "lb_expr.cuh"
#include "kquad_tables.h"

namespace lb {

__device__ __forceinline__ double warp_max(double a) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  return a;
}
__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

// log of the prefactor sqrt(pi) e^{-x} / (Gamma(v+1/2) (2x)^v)
__device__ __forceinline__ double kint_prefactor(double v, double x) {
  return kHalfLogPi - lgamma(v + 0.5) - fma(v, fm_log(2.0 * x), x);
}

// Warp-cooperative Gauss-rule evaluation; every lane returns the same value.
// All 32 lanes must call it with the same (v, x).
//   DX = false: log int_0^inf F(s) ds.
//   DX = true:  d/dx log int_0^inf F(s) ds = (2v - 1) <1/(s + 2x)>_F, the
//               F-weighted mean over the same nodes (dF/dx = F (2v-1)/(s+2x)).
template <bool DX>
__device__ __forceinline__ double kint_gauss(double v, double x, int lane) {
  const double beta = 16.0 / (2.0 * v + 1.0);
  const double logbeta = fm_log(beta);
  const double vm = v - 0.5, tx = 2.0 * x;
  // g piece
  const double* gu;
  const double* gw;
  int ng;
  if (v >= 0.9 || x >= 0.25) { gu = lb_kq_g32_logu; gw = lb_kq_g32_logw; ng = 32; }
  else if (v >= 0.4 || x >= 1e-3) { gu = lb_kq_g64_logu; gw = lb_kq_g64_logw; ng = 64; }
  else { gu = lb_kq_g128_logu; gw = lb_kq_g128_logw; ng = 128; }
  // h piece
  const double *hs, *hy, *hc;
  int nh;
  if (v <= 1.2) { hs = lb_kq_hl32_s; hy = lb_kq_hl32_y; hc = lb_kq_hl32_c; nh = 32; }
  else if (v <= 5.0) { hs = lb_kq_hl48_s; hy = lb_kq_hl48_y; hc = lb_kq_hl48_c; nh = 48; }
  else { hs = lb_kq_hq32_s; hy = lb_kq_hq32_y; hc = lb_kq_hq32_c; nh = 32; }
  // Up to 4 g terms and 2 h terms per lane; the node counts are the same on
  // every lane, so these branches never diverge.
  double L[6], A[6];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = lane + 32 * k;
    L[k] = -INFINITY;
    A[k] = 0.0;
    if (32 * k < ng) {
      const double logu = __ldg(gu + j);
      const double ub = fm_exp(beta * logu);
      L[k] = __ldg(gw + j) + logbeta - ub + fma(vm, fm_log(tx + ub), 7.0 * logu);
      if (DX) A[k] = 1.0 / (tx + ub);
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = lane + 32 * k;
    L[4 + k] = -INFINITY;
    A[4 + k] = 0.0;
    if (j < nh) {
      const double sj = __ldg(hs + j);
      L[4 + k] = fma(vm, __ldg(hy + j) + fm_log(sj + tx), __ldg(hc + j));
      if (DX) A[4 + k] = 1.0 / (sj + tx);
    }
  }
  double m = L[0];
#pragma unroll
  for (int i = 1; i < 6; ++i) m = fmax(m, L[i]);
  m = warp_max(m);
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const bool live = (k < 4) ? (32 * k < ng) : (32 * (k - 4) < nh && L[k] > -INFINITY);
    if (live) {
      const double e = fm_exp(L[k] - m);
      s0 += e;
      if (DX) s1 = fma(e, A[k], s1);
    }
  }
  s0 = warp_sum(s0);
  if (DX) {
    s1 = warp_sum(s1);
    return (2.0 * v - 1.0) * (s1 / s0);
  }
  return m + fm_log(s0);
}

// Warp-cooperative log int_0^1 (g + h) du by the paper's Simpson rule (N = 600).
__device__ __forceinline__ double kint_log_simpson(double v, double x, int lane) {
  const int N = 600;
  const double beta = 16.0 / (2.0 * v + 1.0);
  const double logbeta = log(beta);
  const double vm = v - 0.5, tx = 2.0 * x;
  const double a2 = 2.0 * v + 1.0;
  // heuristic maxima: g at u = 1, h at u* = 1/2 (v < 2) or 1/(2v)
  const double mg = logbeta - 1.0 + vm * log(tx + 1.0);
  const double us = (v < 2.0) ? 0.5 : 0.5 / v;
  const double mh = -1.0 / us - a2 * log(us) + vm * log1p(tx * us);
  double sg = 0.0, sh = 0.0;
  for (int k = lane + 1; k <= N; k += 32) {
    const double u = (double)k / (double)N;
    const double w = (k == N) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
    const double lu = log(u);
    const double ub = exp(beta * lu);
    const double lg = logbeta - ub + fma(vm, log(tx + ub), 7.0 * lu);
    const double lh = -1.0 / u - a2 * lu + vm * log1p(tx * u);
    sg = fma(w, exp(lg - mg), sg);
    sh = fma(w, exp(lh - mh), sh);
  }
  sg = warp_sum(sg);
  sh = warp_sum(sh);
  const double lG = mg + log(sg), lH = mh + log(sh);
  const double M = fmax(lG, lH);
  return M + log(exp(lG - M) + exp(lH - M)) - log(3.0 * N);
}

}  // namespace lb
