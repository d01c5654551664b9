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
//   LB_TIGHT: Gauss rules (tables in kquad_tables.h).  Values (not the
//     x-derivative) for 2 <= v <= 16.5: one lane slot, the split moved from
//     s = 1 to s0 (kint_sum_one).  Otherwise, for 1.2 < v <= 5: 24
//     g nodes and 40 h nodes (two full lane slots).  Otherwise g: Gauss-Legendre in u
//     with 32 nodes (v >= 0.9 or x >= 0.25), 64 (v >= 0.4 or x >= 1e-3), or
//     for v < 0.4, x < 1e-3 a split rule (kint_sums_split), because
//     (2x + u^beta)^(v-1/2) turns sharply near u = (2x)^(1/beta).  h: Gauss-Legendre in log s on
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
#include "lb_intmath.cuh"
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
  return kHalfLogPi - lgamma(v + 0.5) - fma(v, ix_log(2.0 * x), x);
}

// Node counts of the tight rule for one pair, packed as (g rule) | (h rule << 8):
// g rule 32 / 64 = Gauss-Legendre in u with that many nodes, 0 = the split
// rule for small orders and tiny arguments (below); h rule 0 = Gauss-Legendre
// in log s with 32 nodes, 1 = with 48, 2 = Gauss-Laguerre 32.
// g rule 24 goes with h rule 3 (40 nodes in log s): for 1.2 < v <= 5 the
// 24 + 40 nodes fill two 32-lane slots (the 32 + 48 of the general rule take
// three), error map below 4e-17 over x in [1e-300, 30].
// h rules 4, 5 and 6 are the one-slot rules of kint_sum_one (22 g + 10 h
// nodes, s0 = 8, for 2 <= v < 7; 12 + 20, s0 = 3, for 7 <= v <= 16.5;
// 24 + 8, s0 = 10 and n = 6 (beta = 12/(2v+1)), for 0.9 <= v < 2 and
// x >= 0.8), for values and x-derivatives: their error maps (30-digit sums
// of the double tables against the oracle) stay below 1.5e-17 of the error
// scale for log K (over x in [1e-300, 30]; [0.8, 30] for rule 6) and below
// 1.1e-16 relative (the reference's own rounding) for d/dx log K.
// The x-derivative, a weighted mean of 1/(s + 2x) over the nodes, moves both
// boundaries up for v < 0.1: 64 g nodes up to x = 0.6 and the split rule up
// to x = 5e-3.  There the 32-node rule leaves up to 7e-15 relative error in
// the derivative (v = 0, x = 0.25) and the 64-node rule 8e-15 (v = 0,
// x = 1e-3); the rules taken instead stay below 1.2e-16 (error map of the
// derivative rules against the oracle's Bessel ratio).
// (v, x >= 0: the compares run on the bit patterns, integer instructions.)
__device__ __forceinline__ int kint_rule(double v, double x, bool dx) {
  if (LB_GE(v, 2.0) && LB_LE(v, 16.5)) return LB_LT(v, 7.0) ? (22 | (4 << 8)) : (12 | (5 << 8));
  if (LB_GE(v, 0.9) && LB_LT(v, 2.0) && LB_GE(x, 0.8)) return 24 | (6 << 8);
  if (LB_GT(v, 1.2) && LB_LE(v, 5.0)) return 24 | (3 << 8);
  const bool dsmall = dx && LB_LT(v, 0.1);
  const double x32 = dsmall ? 0.6 : 0.25, xsplit = dsmall ? 5e-3 : 1e-3;
  const int ng = (LB_GE(v, 0.9) || LB_GE(x, x32)) ? 32 : ((LB_GE(v, 0.4) || LB_GE(x, xsplit)) ? 64 : 0);
  const int hr = LB_LE(v, 1.2) ? 0 : (LB_LE(v, 5.0) ? 1 : 2);
  return ng | (hr << 8);
}

// Code path of a pair's rule, for sorting pairs by rule: 0 the split rule,
// 1 the one-slot rules with s0 = 8 and s0 = 10, 2 the one-slot rule with
// s0 = 3, 3 the packed rule, 4 and 5 the fixed rules with 32 and 64 g nodes.
__device__ __forceinline__ int kint_class(double v, double x, bool dx) {
  const int rule = kint_rule(v, x, dx);
  const int ng = rule & 0xff, hr = rule >> 8;
  if (ng == 0) return 0;
  if (hr >= 4) return hr == 5 ? 2 : 1;
  return ng == 24 ? 3 : (ng == 32 ? 4 : 5);
}

// One order for every pair of a call (v_stride 0): the g-node positions
// u_j^beta of the three u rules and the order's part of the prefactor are
// the same for every pair, so a block computes them once (with the same
// operations as the per-pair path: the results do not change).
struct KintScalar {
  double ub24[24], ub32[32], ub64[64];
  double sg[24];                                   // s0 u_j^beta of the one-slot rule of v (if any)
  long long ubq24[24], ubq32[32], ubq64[64], sgq[24];   // the same in Q53 (values' fixed-point terms)
  double pre;                                      // log(sqrt(pi)) - lgamma(v + 1/2)
};

// All threads of the block call it; ends with a barrier.
__device__ __forceinline__ void kint_scalar_setup(KintScalar& ks, double v) {
  const int tid = threadIdx.x;
  const double beta = 16.0 * ix_rcp(2.0 * v + 1.0);       // as in kint_batch_gauss
  if (tid < 24) {
    ks.ub24[tid] = ix_exp(beta * __ldg(lb_kq_g24_logu + tid));
    ks.ubq24[tid] = ix_fix(ks.ub24[tid], 53);
  } else if (tid < 56) {
    ks.ub32[tid - 24] = ix_exp(beta * __ldg(lb_kq_g32_logu + tid - 24));
    ks.ubq32[tid - 24] = ix_fix(ks.ub32[tid - 24], 53);
  } else if (tid < 120) {
    ks.ub64[tid - 56] = ix_exp(beta * __ldg(lb_kq_g64_logu + tid - 56));
    ks.ubq64[tid - 56] = ix_fix(ks.ub64[tid - 56], 53);
  } else if (tid == 120) {
    ks.pre = kHalfLogPi - lgamma(v + 0.5);
  } else if (tid >= 128 && tid < 152) {
    const int j = tid - 128;
    bool set = true;
    if (v >= 2.0 && v <= 16.5 && v < 7.0 && j < 22) ks.sg[j] = ix_exp(fma(beta, __ldg(lb_kq_g22_logu + j), LB_KQ_LOG8));
    else if (v >= 7.0 && v <= 16.5 && j < 12) ks.sg[j] = ix_exp(fma(beta, __ldg(lb_kq_g12_logu + j), LB_KQ_LOG3));
    else if (v >= 0.9 && v < 2.0)                  // the rule with n = 6 (beta = 12/(2v+1))
      ks.sg[j] = ix_exp(fma(0.75 * beta, __ldg(lb_kq_g24_logu + j), LB_KQ_LOG10));
    else set = false;
    if (set) ks.sgq[j] = ix_fix(ks.sg[j], 53);
  }
  __syncthreads();
}

// Warp sum of values below 2^63 (the result must stay below 2^64), exact,
// on the integer pipe: three limbs of 20, 20 and 23 bits, one warp
// reduction each (a limb sum stays below 2^28).
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t t) {
  const unsigned a0 = __reduce_add_sync(0xffffffffu, (unsigned)(t & 0xfffffu));
  const unsigned a1 = __reduce_add_sync(0xffffffffu, (unsigned)(t >> 20) & 0xfffffu);
  const unsigned a2 = __reduce_add_sync(0xffffffffu, (unsigned)(t >> 40));
  return (uint64_t)a0 + ((uint64_t)a1 << 20) + ((uint64_t)a2 << 40);
}

// Values (not the x-derivative) with the fixed, packed and one-slot rules.
// Each node's log term L = C - S + (v - 1/2)(Y + log z) -- C the table
// constant (plus the pair's gk for g nodes: log beta, and (v + 1/2) log s0
// for the one-slot rules), Y = log s for h nodes, S = s for g nodes,
// z = s + 2x -- is shifted by mm, the exact warp maximum of L, and the terms
// e^(L - mm) are formed in Q58 (Q56 where a lane holds up to four terms)
// and summed exactly on the integer pipe.
//   FX (pairs with v <= 16.5, x <= 32: the K integral's whole domain in
//   every dispatch): L, its maximum and the shift are Q53 fixed point
//   (lb_intmath.cuh): integer instructions from log z to the Q58 term, with
//   no double packed or unpacked between the steps.  The FP64 pipe does only
//   z = s + 2x (and, with one order per pair, the g nodes' beta log u_j).
//   |L| stays below 2^8 there, inside Q53's 2^10.
//   !FX (a forced evaluation far outside, logbessel_eval_region): L as a
//   double, whatever its size.

// Warp maximum of signed 64-bit integers: the maximum high word (signed),
// then the maximum low word (unsigned) among the lanes that hold it.
__device__ __forceinline__ long long warp_max_i64(long long k) {
  const int khi = (int)(k >> 32);
  const int mhi = __reduce_max_sync(0xffffffffu, khi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, khi == mhi ? (unsigned)k : 0u);
  return (long long)(((unsigned long long)(unsigned)mhi << 32) | mlo);
}

// A double mapped to an int64 of the same order (negative values with all
// but the sign bit flipped), and back.
__device__ __forceinline__ long long key64(double a) {
  const long long b = __double_as_longlong(a);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double key64_to_double(long long m) {
  return __longlong_as_double(m ^ ((m >> 63) & 0x7fffffffffffffffll));
}

// One node's log term in Q53 (vmq = v - 1/2 in Q58).
__device__ __forceinline__ long long kq_term(long long vmq, double z, long long Y, long long C, long long S) {
  return C - S + ix_mul_q58(vmq, Y + ix_log_q53(z));
}

// The pair's arguments of a values sum, broadcast to the warp: v - 1/2 and
// gk in Q53/Q58 (FX) or as doubles, 2x, beta (g nodes per pair only).
struct KqPair {
  long long vmq, gkq;
  double vm, gk, tx, beta;
};

template <bool FX> struct KqLog { typedef double type; };
template <> struct KqLog<true> { typedef long long type; };

// A node's operands: z = s + 2x, and Y, C, S of its log term (in Q53 for
// FX, as doubles y, c, s otherwise).  Lanes that hold g nodes and lanes that
// hold h nodes of the same slot select their operands and then share one
// evaluation (kq_eval), so a warp runs the logarithm once per slot.
struct KqNode {
  double z, y, c, s;
  long long Y, C, S;
};

// A g node: position s = e^(beta log u_j + log s0) per pair, or s from the
// block's table (tab, tabq) with one order per call.
template <bool FX>
__device__ __forceinline__ KqNode kq_g(const KqPair& p, double logu, double logs0, const double* tab,
                                       const long long* tabq, int j, const double* c, const long long* cq) {
  KqNode n;
  const double s = tab ? tab[j] : ix_exp(fma(p.beta, logu, logs0));
  n.z = p.tx + s;
  if constexpr (FX) {
    n.S = tab ? tabq[j] : ix_fix(s, 53);
    n.Y = 0;
    n.C = __ldg(cq + j) + p.gkq;
  } else {
    n.s = s;
    n.y = 0.0;
    n.c = __ldg(c + j) + p.gk;
  }
  return n;
}

// An h node (tables s, y, c; y and c also in Q53).
template <bool FX>
__device__ __forceinline__ KqNode kq_h(const KqPair& p, const double* hs, const double* hy, const long long* hyq,
                                       const double* hc, const long long* hcq, int j) {
  KqNode n;
  n.z = __ldg(hs + j) + p.tx;
  if constexpr (FX) {
    n.S = 0;
    n.Y = __ldg(hyq + j);
    n.C = __ldg(hcq + j);
  } else {
    n.s = 0.0;
    n.y = __ldg(hy + j);
    n.c = __ldg(hc + j);
  }
  return n;
}

// The node's log term C - S + (v - 1/2)(Y + log z).
template <bool FX>
__device__ __forceinline__ typename KqLog<FX>::type kq_eval(const KqPair& p, const KqNode& n) {
  if constexpr (FX) return kq_term(p.vmq, n.z, n.Y, n.C, n.S);
  else return fma(p.vm, ix_log(n.z) + n.y, n.c) - n.s;
}

// Order key of a log term for the warp maximum, the maximum from the
// maximum key, and a term e^(L - mm) in Q58.
template <bool FX> __device__ __forceinline__ long long kq_key(typename KqLog<FX>::type L) {
  if constexpr (FX) return L; else return key64(L);
}
template <bool FX> __device__ __forceinline__ typename KqLog<FX>::type kq_max(long long key) {
  if constexpr (FX) return warp_max_i64(key); else return key64_to_double(warp_max_i64(key));
}
template <bool FX>
__device__ __forceinline__ uint64_t kq_exp(typename KqLog<FX>::type L, typename KqLog<FX>::type mm) {
  if constexpr (FX) return ix_exp_q58_fx(L - mm); else return ix_exp_q58(L - mm);
}

// W (the x-derivative): also w1 = sum_j t_j / (s_j + 2x) over the lane's
// terms t_j (the Q58 or Q56 integers, as doubles), so that the F-weighted
// mean of 1/(s + 2x) is w1 / (the integer sum).
template <bool FX, bool W = false>
__device__ __forceinline__ uint64_t kint_sumq_fixed(const KqPair& p, int ng, int hr, int lane,
                                                    typename KqLog<FX>::type& mm, const KintScalar* ks,
                                                    double* w1 = nullptr) {
  typedef typename KqLog<FX>::type LT;
  const double* gu = ng == 32 ? lb_kq_g32_logu : lb_kq_g64_logu;
  const double* gc = ng == 32 ? lb_kq_g32_c : lb_kq_g64_c;
  const long long* gcq = ng == 32 ? lb_kq_g32_c_q : lb_kq_g64_c_q;
  const double* hs = hr == 0 ? lb_kq_hl32_s : (hr == 1 ? lb_kq_hl48_s : lb_kq_hq32_s);
  const double* hy = hr == 0 ? lb_kq_hl32_y : (hr == 1 ? lb_kq_hl48_y : lb_kq_hq32_y);
  const long long* hyq = hr == 0 ? lb_kq_hl32_y_q : (hr == 1 ? lb_kq_hl48_y_q : lb_kq_hq32_y_q);
  const double* hc = hr == 0 ? lb_kq_hl32_c : (hr == 1 ? lb_kq_hl48_c : lb_kq_hq32_c);
  const long long* hcq = hr == 0 ? lb_kq_hl32_c_q : (hr == 1 ? lb_kq_hl48_c_q : lb_kq_hq32_c_q);
  const int nh = hr == 1 ? 48 : 32;
  const double* gtab = ks ? (ng == 32 ? ks->ub32 : ks->ub64) : nullptr;
  const long long* gtabq = ks ? (ng == 32 ? ks->ubq32 : ks->ubq64) : nullptr;
  LT L[4];
  double A[4];                                     // W: 1/(s + 2x)
  long long key = (long long)0x8000000000000000ull;   // below every key
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    L[k] = 0;
    if (32 * k < ng) {
      const int j = lane + 32 * k;
      const KqNode n = kq_g<FX>(p, __ldg(gu + j), 0.0, gtab, gtabq, j, gc, gcq);
      L[k] = kq_eval<FX>(p, n);
      if (W) A[k] = ix_rcp(n.z);
      key = max(key, kq_key<FX>(L[k]));
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = lane + 32 * k;
    L[2 + k] = 0;
    if (j < nh) {
      const KqNode n = kq_h<FX>(p, hs, hy, hyq, hc, hcq, j);
      L[2 + k] = kq_eval<FX>(p, n);
      if (W) A[2 + k] = ix_rcp(n.z);
      key = max(key, kq_key<FX>(L[2 + k]));
    }
  }
  mm = kq_max<FX>(key);
  uint64_t q = 0;
  double w = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool live = (k < 2) ? (32 * k < ng) : (lane + 32 * (k - 2) < nh);
    if (live) {
      const uint64_t t = kq_exp<FX>(L[k], mm) >> 2;
      q += t;
      if (W) w = fma(__ull2double_rn(t), A[k], w);
    }
  }
  if (W) *w1 = w;
  return warp_sum_u64(q);
}

template <bool FX, bool W = false>
__device__ __forceinline__ uint64_t kint_sumq_g24h40(const KqPair& p, int lane, typename KqLog<FX>::type& mm,
                                                     const KintScalar* ks, double* w1 = nullptr) {
  typedef typename KqLog<FX>::type LT;
  const KqNode n0 = lane < 24 ? kq_g<FX>(p, __ldg(lb_kq_g24_logu + lane), 0.0, ks ? ks->ub24 : nullptr,
                                         ks ? ks->ubq24 : nullptr, lane, lb_kq_g24_c, lb_kq_g24_c_q)
                              : kq_h<FX>(p, lb_kq_hl40_s, lb_kq_hl40_y, lb_kq_hl40_y_q, lb_kq_hl40_c, lb_kq_hl40_c_q,
                                         lane - 24);
  const KqNode n1 = kq_h<FX>(p, lb_kq_hl40_s, lb_kq_hl40_y, lb_kq_hl40_y_q, lb_kq_hl40_c, lb_kq_hl40_c_q, lane + 8);
  const LT L0 = kq_eval<FX>(p, n0);
  const LT L1 = kq_eval<FX>(p, n1);
  mm = kq_max<FX>(max(kq_key<FX>(L0), kq_key<FX>(L1)));
  const uint64_t t0 = kq_exp<FX>(L0, mm) >> 2, t1 = kq_exp<FX>(L1, mm) >> 2;
  if (W) *w1 = fma(__ull2double_rn(t0), ix_rcp(n0.z), __ull2double_rn(t1) * ix_rcp(n1.z));
  return warp_sum_u64(t0 + t1);
}

// One pair, one lane slot (values, 2 <= v <= 16.5).  int_0^inf F(s) ds is
// split at s0 instead of 1: on [s0, inf), t = s - s0, the branch point s = 0
// of (s (s + 2x))^(v-1/2) is s0 away from the Gauss-Laguerre nodes, so 10
// or 20 of them reach 1e-17; [0, s0] takes s = s0 u^beta and Gauss-Legendre
// in u on the remaining lanes.  A g node's constant is c + gk with
// gk = (v+1/2) log s0 + log beta (per pair), an h node's c (with -s0 folded
// in) and Y = log s.  Rule 4: s0 = 8, 22 g + 10 h nodes (2 <= v < 7);
// rule 5: s0 = 3, 12 + 20 (7 <= v <= 16.5).  Error map against a 34-digit
// reference, over x in [1e-300, 30]: below 1.5e-17 of the error scale
// max(1, |x d/dx log K|, |v d/dv log K|).  Returns the sum, on every lane,
// in Q58.
template <bool FX, bool W = false>
__device__ __forceinline__ uint64_t kint_sum_one(const KqPair& p, int hr, int lane, typename KqLog<FX>::type& mm,
                                                 const KintScalar* ks, double* w1 = nullptr) {
  typedef typename KqLog<FX>::type LT;
  const bool r4 = hr == 4, r6 = hr == 6;
  const int ng = r4 ? 22 : (r6 ? 24 : 12);
  const double* gu = r4 ? lb_kq_g22_logu : (r6 ? lb_kq_g24_logu : lb_kq_g12_logu);
  const double* gc = r4 ? lb_kq_g22_c : (r6 ? lb_kq_g24n6_c : lb_kq_g12_c);
  const long long* gcq = r4 ? lb_kq_g22_c_q : (r6 ? lb_kq_g24n6_c_q : lb_kq_g12_c_q);
  const double ls0 = r4 ? LB_KQ_LOG8 : (r6 ? LB_KQ_LOG10 : LB_KQ_LOG3);
  const double* hs = r4 ? lb_kq_hq10o8_s : (r6 ? lb_kq_hq8o10_s : lb_kq_hq20o3_s);
  const double* hy = r4 ? lb_kq_hq10o8_y : (r6 ? lb_kq_hq8o10_y : lb_kq_hq20o3_y);
  const long long* hyq = r4 ? lb_kq_hq10o8_y_q : (r6 ? lb_kq_hq8o10_y_q : lb_kq_hq20o3_y_q);
  const double* hc = r4 ? lb_kq_hq10o8_c : (r6 ? lb_kq_hq8o10_c : lb_kq_hq20o3_c);
  const long long* hcq = r4 ? lb_kq_hq10o8_c_q : (r6 ? lb_kq_hq8o10_c_q : lb_kq_hq20o3_c_q);
  const KqNode n = lane < ng ? kq_g<FX>(p, __ldg(gu + lane), ls0, ks ? ks->sg : nullptr, ks ? ks->sgq : nullptr,
                                        lane, gc, gcq)
                             : kq_h<FX>(p, hs, hy, hyq, hc, hcq, lane - ng);
  const LT L = kq_eval<FX>(p, n);
  mm = kq_max<FX>(kq_key<FX>(L));
  const uint64_t t = kq_exp<FX>(L, mm);
  if (W) *w1 = __ull2double_rn(t) * ix_rcp(n.z);
  return warp_sum_u64(t);
}

// The pairs of one values rule group (lanes in grp), one at a time: the
// pair's arguments broadcast from its lane, its sum by the warp, and the
// sum and shift kept on its lane.
// W (the x-derivative): also the warp sum of the weighted terms, in s1_i.
template <bool FX, int CLS, bool W = false>
__device__ __forceinline__ void kint_q_group(unsigned grp, int ng, int hr, int lane, long long vmq_i, long long gkq_i,
                                             double vm_i, double gk_i, double tx_i, double beta_i, double& m_i,
                                             long long& mq_i, uint64_t& q_i, const KintScalar* ks,
                                             double* s1_i = nullptr) {
  for (; grp; grp &= grp - 1) {
    const int e = __ffs(grp) - 1;
    KqPair p;
    if constexpr (FX) {
      p.vmq = __shfl_sync(0xffffffffu, vmq_i, e);
      p.gkq = __shfl_sync(0xffffffffu, gkq_i, e);
    } else {
      p.vm = __shfl_sync(0xffffffffu, vm_i, e);
      p.gk = __shfl_sync(0xffffffffu, gk_i, e);
    }
    p.tx = __shfl_sync(0xffffffffu, tx_i, e);
    p.beta = ks ? 0.0 : __shfl_sync(0xffffffffu, beta_i, e);
    typename KqLog<FX>::type mm = 0;
    uint64_t q = 0;
    double w = 0.0;
    if constexpr (W) {                             // the derivative: one-slot, packed and fixed rules
      if constexpr (CLS == 1 || CLS == 2) {
        q = kint_sum_one<FX, true>(p, hr, lane, mm, ks, &w);
      } else if constexpr (CLS == 3) {
        q = kint_sumq_g24h40<FX, true>(p, lane, mm, ks, &w);
      } else if constexpr (CLS == 4 || CLS == 5) {
        q = kint_sumq_fixed<FX, true>(p, ng, hr, lane, mm, ks, &w);
      } else {
        if (hr >= 4) q = kint_sum_one<FX, true>(p, hr, lane, mm, ks, &w);
        else if (ng == 24) q = kint_sumq_g24h40<FX, true>(p, lane, mm, ks, &w);
        else q = kint_sumq_fixed<FX, true>(p, ng, hr, lane, mm, ks, &w);
      }
      w = warp_sum(w);
    } else if constexpr (CLS == 1 || CLS == 2) {
      q = kint_sum_one<FX>(p, hr, lane, mm, ks);
    } else if constexpr (CLS == 3) {
      q = kint_sumq_g24h40<FX>(p, lane, mm, ks);
    } else if constexpr (CLS == 4 || CLS == 5) {
      q = kint_sumq_fixed<FX>(p, ng, hr, lane, mm, ks);
    } else if constexpr (CLS < 0) {
      if (hr >= 4) q = kint_sum_one<FX>(p, hr, lane, mm, ks);
      else if (ng == 24) q = kint_sumq_g24h40<FX>(p, lane, mm, ks);
      else q = kint_sumq_fixed<FX>(p, ng, hr, lane, mm, ks);
    }
    if (lane == e) {
      if constexpr (FX) mq_i = mm;                 // to a double once, after the batch
      else m_i = mm;
      q_i = q;
      if constexpr (W) *s1_i = w;
    }
  }
}

// Split g rule (v < 0.4, x < 1e-3).  (2x + u^beta)^(v-1/2) turns within a
// width ~1/beta of u = (2x)^(1/beta), and for v -> 0 the integrand is
// log-uniform between s ~ 2x and 1, which no fixed rule in u resolves as
// x -> 0.  So int_0^1 F(s) ds is split at s1 = 128 x:
//   [0, s1]: s = s1 u^beta, the 64-node Gauss-Legendre rule in u (the turn
//            now sits at u^beta = 1/64, where that rule is exact to 1e-16);
//   [s1, 1]: y = log s, F(s) s = e^{-s} s^(v+1/2) (s + 2x)^(v-1/2), with
//            Gauss-Legendre panels [y1, y1 + 8] (16 nodes) and
//            [y1 + 8, y1 + 40] (32) for the tail of the turn (y1 = log s1),
//            [-40, -4] (32) and [-4, 0] (16) for the e^{-s} roll-off, each
//            cut where it meets the next; in between, F(s) s = e^{2 v y} to
//            1e-17 and is integrated in closed form.
// The nodes of [0, s1] and of the two panels that start at y1 are placed by
// their offset o = y - y1 (s = s1 e^o), and their log terms are kept less the
// common part C = 2 v y1 (log(s + 2x) = y1 + log(e^o + 1/64)): so the
// hundreds-sized y1 never enters a node's term, whose rounding would
// otherwise shift each node by ~|y1| ulp and cost the x-derivative (a
// weighted mean of 1/(s + 2x) over the nodes) two digits.  These terms are
// shifted by mm - C instead of mm.  Slots: 0, 1 the 64 nodes of [0, s1];
// 2 = two 16-node panels ([y1, y1 + 8] on lanes 0-15, [-4, 0] on 16-31);
// 3 = [y1 + 8, y1 + 40]; 4 = [-40, -4]; 5 = the 32 h nodes (v < 0.4, so h
// is the 32-node rule in log s).
template <bool DX>
__device__ __forceinline__ void kint_sums_split(double v, double x, double beta, int lane,
                                                double& mm, double& s0, double& s1, const KintScalar* ks) {
  const double vm = v - 0.5, vp = v + 0.5, tx = 2.0 * x;
  const double sx = 128.0 * x;                     // s1 (exact)
  const double y1 = ix_log(sx);
  const double C = 2.0 * v * y1;
  double L[6], A[6];
  bool live[6], rel[6];
  int key = (int)0x800fffff;
#pragma unroll
  for (int k = 0; k < 2; ++k) {                    // [0, s1]: s = s1 r, r = u^beta
    const int j = lane + 32 * k;
    const double r = ks ? ks->ub64[j] : ix_exp(beta * __ldg(lb_kq_g64_logu + j));
    const double sj = sx * r;
    L[k] = fma(vm, ix_log(r + 0.015625), __ldg(lb_kq_g64_c + j)) - sj;     // less log beta, as above
    A[k] = DX ? ix_rcp(sj + tx) : 0.0;
    live[k] = true;
    rel[k] = true;
    key = max(key, order_key(L[k] + C));
  }
#pragma unroll
  for (int k = 2; k < 5; ++k) {
    double a, b, t, lw;
    bool anchored;
    if (k == 2) {
      const int j = lane & 15;
      t = __ldg(lb_kq_gl16_t + j);
      lw = __ldg(lb_kq_gl16_logw + j);
      anchored = lane < 16;
      if (anchored) { a = 0.0; b = fmin(8.0, -4.0 - y1); }       // offsets
      else { a = fmax(y1, -4.0); b = 0.0; }
    } else {
      t = __ldg(lb_kq_gl32_t + lane);
      lw = __ldg(lb_kq_gl32_logw + lane);
      anchored = k == 3;
      if (anchored) { a = 8.0; b = fmin(40.0, -4.0 - y1); }       // offsets
      else { a = fmax(y1 + 40.0, -40.0); b = -4.0; }
    }
    live[k] = b > a;
    rel[k] = anchored;
    L[k] = 0.0;
    A[k] = 0.0;
    if (live[k]) {
      const double o = fma(b - a, t, a);
      const double lwb = lw + ix_log(b - a);
      double sj;
      if (anchored) {                              // y = y1 + o
        const double eo = ix_exp(o);
        sj = sx * eo;
        L[k] = fma(vm, ix_log(eo + 0.015625), fma(vp, o, lwb)) - sj;
        key = max(key, order_key(L[k] + C));
      } else {                                     // y = o
        sj = ix_exp(o);
        L[k] = fma(vm, ix_log(sj + tx), fma(vp, o, lwb)) - sj;
        key = max(key, order_key(L[k]));
      }
      if (DX) A[k] = ix_rcp(sj + tx);
    }
  }
  {                                                // h nodes, 32-node rule in log s
    const double sj = __ldg(lb_kq_hl32_s + lane);
    L[5] = fma(vm, __ldg(lb_kq_hl32_y + lane) + ix_log(sj + tx), __ldg(lb_kq_hl32_c + lane));
    A[5] = DX ? ix_rcp(sj + tx) : 0.0;
    live[5] = true;
    rel[5] = false;
    key = max(key, order_key(L[5]));
  }
  // flat middle [y1 + 40, -40]: int e^{2 v y} dy = e^{2 v (y1 + 40)} (e^{2 v w} - 1) / (2 v), w = -80 - y1;
  // less C: 80 v + log(expm1(2 v w) / (2 v))
  const double w = -80.0 - y1;
  const bool flat = w > 0.0;
  double Lflat = 0.0;
  if (flat) {
    Lflat = (v == 0.0) ? fm_log(w) : fma(80.0, v, fm_log(expm1(2.0 * v * w) / (2.0 * v)));
    key = max(key, order_key(Lflat + C));
  }
  mm = key_to_double(__reduce_max_sync(0xffffffffu, key));
  const double mr = mm - C;
  double g0 = 0.0, g1 = 0.0;
  s0 = 0.0;
  s1 = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (live[k]) {
      const double t = ix_exp(L[k] - (rel[k] ? mr : mm));
      if (k < 2) {
        g0 += t;
        if (DX) g1 = fma(t, A[k], g1);
      } else {
        s0 += t;
        if (DX) s1 = fma(t, A[k], s1);
      }
    }
  }
  s0 = fma(beta, g0, s0);
  if (DX) s1 = fma(beta, g1, s1);
  if (flat && lane == 0) {
    s0 += ix_exp(Lflat - mr);
    if (DX) {
      // there 1/(s + 2x) = e^{-y} to 1e-17: int e^{(2v-1) y} dy over the same
      // interval, less C: (2v - 1) 40 - y1 + log((1 - e^{(2v-1) w}) / (1 - 2v))
      const double c = 2.0 * v - 1.0;
      s1 += ix_exp(fma(40.0, c, -y1) + fm_log(-expm1(c * w) / -c) - mr);
    }
  }
}

// K integrals of up to 32 pairs by one warp (Gauss rules; lane e holds pair
// e, all lanes pass valid data).  Per pair, the lanes split the nodes; the
// log-sum-exp shift is the warp maximum taken on the integer pipe, the sum a
// warp-shuffle reduction (Eq. "log sum trick").  Everything that is per pair
// rather than per node (the order-dependent constants, the prefactor, the
// final logarithm) is computed once per lane for its own pair, not once per
// pair by all 32 lanes.  The rule is uniform across the warp for each pair,
// so the split and fixed paths never diverge.  Returns, on lane e, log K of
// pair e (DX = false) or d/dx log K (DX = true: the prefactor derivative
// -v/x - 1 plus (2v - 1) <1/(s + 2x)>, the F-weighted mean over the nodes,
// since dF/dx = F (2v - 1)/(s + 2x)).
// CLS >= 0: every pair of the batch is of rule class CLS (kint_class), and
// only that class's code is compiled, so a kernel built for one class holds
// the registers of its own rule only.
template <bool DX, int CLS = -1>
__device__ __forceinline__ double kint_batch_gauss(double vi, double xi, int npairs, int lane,
                                                   const KintScalar* ks = nullptr) {
  const int rule_i = kint_rule(vi, xi, DX);
  // beta = 2n/(2v+1): n = 8, or 6 for the one-slot rule of 0.9 <= v < 2
  const double beta_i = ((rule_i >> 8) == 6 ? 12.0 : 16.0) * ix_rcp(2.0 * vi + 1.0);   // reciprocal on the integer pipe
  // values: the g nodes' common factor as a log, log beta (plus
  // (v + 1/2) log s0 = (v - 1/2) log s0 + log s0 for the one-slot rules),
  // added to their log terms; in the fixed-point domain (v <= 16.5, x <= 32)
  // in Q53 with v - 1/2 in Q58, else as doubles
  const bool fx_i = LB_LE(vi, 16.5) && LB_LE(xi, 32.0);
  long long vmq_i = 0, gkq_i = 0;
  double vm_i = 0.0, gk_i = 0.0;
  {
    const int hr_i = rule_i >> 8;
    if (fx_i) {
      vmq_i = ix_fix(vi - 0.5, 58);
      gkq_i = ix_log_q53(beta_i);
      if (hr_i >= 4) {
        const long long ls0 = hr_i == 4 ? LB_KQ_LOG8_Q53 : (hr_i == 6 ? LB_KQ_LOG10_Q53 : LB_KQ_LOG3_Q53);
        gkq_i += ix_mul_q58(vmq_i, ls0) + ls0;
      }
    } else {
      vm_i = vi - 0.5;
      gk_i = ix_log(beta_i);
      if (hr_i >= 4) gk_i = fma(vi + 0.5, hr_i == 4 ? LB_KQ_LOG8 : (hr_i == 6 ? LB_KQ_LOG10 : LB_KQ_LOG3), gk_i);
    }
  }
  const double tx_i = 2.0 * xi;
  double m_i = 0.0, s0_i = 1.0, s1_i = 0.0;
  long long mq_i = 0;                              // the shift of a fixed-point pair, Q53
  uint64_t q_i = 0;                                // fixed-point sum (values, all rules but the split one)
  int qb_i = 0;                                    // its fraction bits
  // The pairs are taken rule by rule (lanes with the same rule found by a
  // ballot), so each rule's code runs for all its pairs of the batch before
  // the next rule's: in a batch that mixes rules, switching code paths at
  // every pair thrashed the instruction cache.  The order of the pairs does
  // not change any result.
  // Pairs outside the fixed-point domain form groups of their own.
  const int key_i = rule_i | (fx_i ? 0 : 1 << 16);
  unsigned rem = npairs >= 32 ? 0xffffffffu : ((1u << npairs) - 1u);
  while (rem) {
    const int key = __shfl_sync(0xffffffffu, key_i, __ffs(rem) - 1);
    unsigned grp = __ballot_sync(0xffffffffu, key_i == key) & rem;
    rem &= ~grp;
    const int rule = key & 0xffff;
    const int ng = rule & 0xff, hr = rule >> 8;
    if (CLS != 0 && ng != 0) {
      const int qb = hr >= 4 ? 58 : 56;
      if ((grp >> lane) & 1u) qb_i = qb;
      if ((key >> 16) == 0)
        kint_q_group<true, CLS, DX>(grp, ng, hr, lane, vmq_i, gkq_i, vm_i, gk_i, tx_i, beta_i, m_i, mq_i, q_i, ks,
                                    &s1_i);
      else
        kint_q_group<false, CLS, DX>(grp, ng, hr, lane, vmq_i, gkq_i, vm_i, gk_i, tx_i, beta_i, m_i, mq_i, q_i, ks,
                                     &s1_i);
      continue;
    }
    for (; grp; grp &= grp - 1) {
      const int e = __ffs(grp) - 1;
      const double v = __shfl_sync(0xffffffffu, vi, e);
      const double x = __shfl_sync(0xffffffffu, xi, e);
      const double beta = __shfl_sync(0xffffffffu, beta_i, e);
      double mm, s0, s1 = 0.0;
      kint_sums_split<DX>(v, x, beta, lane, mm, s0, s1, ks);   // the other rules take the sums above
      s0 = warp_sum(s0);
      if (DX) s1 = warp_sum(s1);
      if (lane == e) {
        m_i = mm;
        s0_i = s0;
        s1_i = s1;
      }
    }
  }
  if (DX) {
    if (qb_i) s0_i = __ull2double_rn(q_i);        // the weighted sum is in the same units
    return -(vi / xi + 1.0) + (2.0 * vi - 1.0) * (s1_i / s0_i);
  }
  if (qb_i) {
    s0_i = __ull2double_rn(q_i) * (qb_i == 58 ? 0x1p-58 : 0x1p-56);   // exact scalings
    if (fx_i) m_i = __ll2double_rn(mq_i) * 0x1p-53;
  }
  const double pre = ks ? ks->pre - fma(vi, ix_log(2.0 * xi), xi) : kint_prefactor(vi, xi);
  return pre + m_i + ix_log(s0_i);
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
