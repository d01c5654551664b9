/*
 * logbessel_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, extended-precision CPU evaluator of log I_v(x), log K_v(x),
 * their x-derivatives and the von Mises-Fisher log-normaliser.  It exists to
 * check the CUDA library and is never part of the product path: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * It computes the plain definitions, not the paper's region-dispatched
 * expressions, so it shares no formula with the GPU path:
 *
 *   log I_v(x): the positive-term power series of I_v (paper Sec. 3.1, the
 *     "infinite series" equation; DLMF 10.25.2), summed in double-double
 *     arithmetic outward from the largest term (paper Eq. "K", the peak index),
 *     every term at every x -- no asymptotic expansion, no integral.
 *   log K_v(x): the integral K_v(x) = int_0^inf exp(-x cosh t) cosh(v t) dt
 *     (DLMF 10.32.9), a positive integrand, by the trapezoid rule in
 *     double-double with step halving until it stops changing.  The
 *     trapezoid rule converges geometrically for analytic integrands that
 *     decay at both ends (Trefethen & Weideman, SIAM Review 56, 2014).  This
 *     is not the Rothwell representation the paper uses for small inputs.
 *   d/dx log I_v(x) = I_{v+1}/I_v + v/x          (DLMF 10.29.2, positive form)
 *   d/dx log K_v(x) = -(K_{v-1}/K_v + v/x)       (DLMF 10.29.2, positive form)
 *   log C_d(k) = (d/2-1) log k - (d/2) log 2pi - log I_{d/2-1}(k)
 *                                               (paper Sec. 6.3, vMF density)
 *
 * Arithmetic: a hand-written double-double type (about 106 bits; Dekker 1971,
 * Knuth TAOCP vol. 2 Sec. 4.2.2, with fma for the exact product).  exp is
 * argument reduction by ln 2 and 2^-10 followed by Taylor and squaring; log is
 * one Newton step on exp from the double log; lgamma is the Stirling series
 * with Bernoulli numbers after an upward shift of the argument (textbook
 * methods, Abramowitz & Stegun 6.1.40).
 *
 * Domain conventions (both the oracle and the library follow them):
 *   I: v < 0 or x < 0 -> NaN; x = 0 -> 0 if v = 0 else -inf; x = +inf -> +inf;
 *      v = +inf (x finite) -> -inf.
 *   K: v -> |v|; x < 0 -> NaN; x = 0 -> +inf; x = +inf -> -inf;
 *      v = +inf (x finite, > 0) -> +inf.
 *   Any NaN input, or v and x both infinite -> NaN.
 * The I evaluators decline arguments x > 1e8 (NaN): the series would need
 * more than ~1e5 terms.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no fast-math).
 */
#define _DEFAULT_SOURCE   /* lgammal_r */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#ifndef ORACLE_LONG_DOUBLE
/* ------------------------------------------------------------------ */
/* double-double arithmetic                                            */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static inline dd dd_make(double hi, double lo) { dd r = {hi, lo}; return r; }
static inline dd dd_from(double a) { return dd_make(a, 0.0); }

static inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd_make(s, e);
}
static inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd_make(s, e);
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd_make(p, e);
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_neg(dd a) { return dd_make(-a.hi, -a.lo); }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static inline dd dd_add_d(dd a, double b) {
  dd s = two_sum(a.hi, b);
  s.lo += a.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_d(b, q2));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add_d(q, q3);
}
static inline dd dd_ldexp(dd a, int e) { return dd_make(ldexp(a.hi, e), ldexp(a.lo, e)); }
static inline dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd_from(a.hi == 0.0 ? 0.0 : NAN);
  double s = sqrt(a.hi);
  dd s2 = two_prod(s, s);
  dd r = dd_sub(a, s2);
  return dd_add_d(dd_from(s), r.hi / (2.0 * s));
}
static inline double dd_to_d(dd a) { return a.hi + a.lo; }

/* ln 2 and pi to double-double precision (published digits:
 * ln 2 = 0.693147180559945309417232121458176568...,
 * pi   = 3.141592653589793238462643383279502884...). */
static const dd DD_LN2 = {6.93147180559945286227e-01, 2.31904681384629955842e-17};
static const dd DD_PI = {3.14159265358979311600e+00, 1.22464679914735320717e-16};

/* 1/k! for k = 0..14 in double-double, filled once before any thread starts. */
static dd INV_FACT[15];
static int inv_fact_ready = 0;
static void init_tables(void) {
  if (inv_fact_ready) return;
  INV_FACT[0] = dd_from(1.0);
  for (int k = 1; k < 15; ++k) INV_FACT[k] = dd_div(INV_FACT[k - 1], dd_from((double)k));
  inv_fact_ready = 1;
}

/* exp(a) for |a| < 709; returns +inf/0 outside. */
static dd dd_exp(dd a) {
  if (a.hi > 709.0) return dd_from(INFINITY);
  if (a.hi < -745.0) return dd_from(0.0);
  double k = nearbyint(a.hi / DD_LN2.hi);
  dd r = dd_sub(a, dd_mul_d(DD_LN2, k));
  r = dd_ldexp(r, -10);                      /* |r| <= 3.4e-4 */
  /* s = exp(r) - 1 = sum_{i=1}^{12} r^i / i! by Horner (r^13/13! < 1e-55) */
  dd s = INV_FACT[12];
  for (int i = 11; i >= 1; --i) s = dd_add(dd_mul(s, r), INV_FACT[i]);
  s = dd_mul(s, r);
  /* exp(2r) - 1 = s (s + 2): square ten times keeping the expm1 form */
  for (int i = 0; i < 10; ++i) s = dd_mul(s, dd_add_d(s, 2.0));
  dd e = dd_add_d(s, 1.0);
  return dd_ldexp(e, (int)k);
}

/* log(1 + t) for |t| < 1e-3 by its Taylor series; else through dd_log. */
static dd dd_log(dd a);
static dd dd_log1p(dd t) {
  if (fabs(t.hi) < 1e-3) {
    dd p = t, s = t;
    for (int i = 2; i <= 16; ++i) {
      p = dd_mul(p, t);
      dd q = dd_div(p, dd_from((double)i));
      s = (i & 1) ? dd_add(s, q) : dd_sub(s, q);
    }
    return s;
  }
  return dd_log(dd_add_d(t, 1.0));
}

/* log(a), a > 0: one Newton step y <- y + a exp(-y) - 1 from the double log. */
static dd dd_log(dd a) {
  if (a.hi <= 0.0) return dd_from(a.hi == 0.0 ? -INFINITY : NAN);
  if (isinf(a.hi)) return dd_from(INFINITY);
  double y0 = log(a.hi);
  dd y = dd_from(y0);
  dd e = dd_exp(dd_neg(y));
  dd c = dd_sub(dd_mul(a, e), dd_from(1.0));
  y = dd_add(y, c);
  /* a second step makes the result independent of the libm log's last bits */
  e = dd_exp(dd_neg(y));
  c = dd_sub(dd_mul(a, e), dd_from(1.0));
  return dd_add(y, c);
}

/* Bernoulli numbers B_2..B_30 (numerator, denominator), published values. */
static const double BERN_NUM[15] = {1.0, -1.0, 1.0, -1.0, 5.0, -691.0, 7.0, -3617.0, 43867.0,
                                    -174611.0, 854513.0, -236364091.0, 8553103.0,
                                    -23749461029.0, 8615841276005.0};
static const double BERN_DEN[15] = {6.0, 30.0, 42.0, 30.0, 66.0, 2730.0, 6.0, 510.0, 798.0,
                                    330.0, 138.0, 2730.0, 6.0, 870.0, 14322.0};

/* lgamma(z) for z >= 1 (double-double argument). */
static dd dd_lgamma(dd z) {
  dd shift_log = dd_from(0.0);
  if (z.hi < 40.0) {
    /* lgamma(z) = lgamma(z + m) - log(z (z+1) ... (z+m-1)) */
    dd prod = dd_from(1.0);
    while (z.hi < 40.0) {
      prod = dd_mul(prod, z);
      z = dd_add_d(z, 1.0);
    }
    shift_log = dd_log(prod);
  }
  /* Stirling: (z-1/2) log z - z + log(2 pi)/2 + sum B_2k / (2k (2k-1) z^(2k-1)) */
  dd lz = dd_log(z);
  dd half_log_2pi = dd_ldexp(dd_log(dd_ldexp(DD_PI, 1)), -1);
  dd res = dd_add(dd_sub(dd_mul(dd_add_d(z, -0.5), lz), z), half_log_2pi);
  dd zinv = dd_div(dd_from(1.0), z);
  dd zinv2 = dd_mul(zinv, zinv);
  dd zp = zinv;
  for (int k = 1; k <= 15; ++k) {
    double den = (2.0 * k) * (2.0 * k - 1.0) * BERN_DEN[k - 1];
    dd c = dd_div(dd_from(BERN_NUM[k - 1]), dd_from(den));
    res = dd_add(res, dd_mul(c, zp));
    zp = dd_mul(zp, zinv2);
  }
  return dd_sub(res, shift_log);
}
#define ORACLE_NOISE_UNIT 1e-31   /* resolution of phi near its peak (double-double) */

#else /* ORACLE_LONG_DOUBLE */
/* ------------------------------------------------------------------ */
/* the same evaluators in the C type long double                       */
/* ------------------------------------------------------------------ */
/* A second build of this file (-DORACLE_LONG_DOUBLE) runs the evaluators
 * below unchanged on the C type long double instead of double-double:
 * binary128 (113-bit significand) on aarch64 Linux, the x87 80-bit format
 * (64-bit significand) on x86-64.  Every double-double operation maps to one
 * long double operation, and exp, log, log1p and lgamma to libm's expl,
 * logl, log1pl and lgammal_r, so the two builds share the algorithm and
 * nothing of the arithmetic: their agreement checks the double-double layer
 * (to ~1e-30 where binary128 exists).  The field lo stays zero. */
typedef long double ldbl;
typedef struct { ldbl hi, lo; } dd;

static inline dd dd_make(ldbl hi, ldbl lo) { dd r = {hi + lo, 0.0L}; return r; }
static inline dd dd_from(double a) { return dd_make((ldbl)a, 0.0L); }
static inline dd two_prod(double a, double b) { return dd_make((ldbl)a * (ldbl)b, 0.0L); }
static inline dd dd_add(dd a, dd b) { return dd_make(a.hi + b.hi, 0.0L); }
static inline dd dd_neg(dd a) { return dd_make(-a.hi, 0.0L); }
static inline dd dd_sub(dd a, dd b) { return dd_make(a.hi - b.hi, 0.0L); }
static inline dd dd_add_d(dd a, double b) { return dd_make(a.hi + (ldbl)b, 0.0L); }
static inline dd dd_mul(dd a, dd b) { return dd_make(a.hi * b.hi, 0.0L); }
static inline dd dd_mul_d(dd a, double b) { return dd_make(a.hi * (ldbl)b, 0.0L); }
static inline dd dd_div(dd a, dd b) { return dd_make(a.hi / b.hi, 0.0L); }
static inline dd dd_ldexp(dd a, int e) { return dd_make(ldexpl(a.hi, e), 0.0L); }
static inline double dd_to_d(dd a) { return (double)a.hi; }

/* ln 2 and pi, the published digits */
static const dd DD_LN2 = {0.693147180559945309417232121458176568L, 0.0L};
static const dd DD_PI = {3.141592653589793238462643383279502884L, 0.0L};

static void init_tables(void) {}

/* the same range as the double-double exp: +inf above 709, 0 below -745 */
static dd dd_exp(dd a) {
  if (a.hi > 709.0L) return dd_from(INFINITY);
  if (a.hi < -745.0L) return dd_from(0.0);
  return dd_make(expl(a.hi), 0.0L);
}
static dd dd_log(dd a) {
  if (a.hi <= 0.0L) return dd_from(a.hi == 0.0L ? -INFINITY : NAN);
  return dd_make(logl(a.hi), 0.0L);
}
static dd dd_log1p(dd t) { return dd_make(log1pl(t.hi), 0.0L); }
static dd dd_lgamma(dd z) {
  int sign;
  return dd_make(lgammal_r(z.hi, &sign), 0.0L);
}

/* resolution of phi near its peak: a few units of the long double epsilon */
#define ORACLE_NOISE_UNIT (8.0 * (double)LDBL_EPSILON)
#endif /* ORACLE_LONG_DOUBLE */

/* ------------------------------------------------------------------ */
/* log I_v(x): positive-term series from the peak term                 */
/* ------------------------------------------------------------------ */
/* v >= 0 (double-double), 0 < x < inf. */
static dd log_i_dd(dd v, double x) {
  const double tiny = 1e-34;
  dd y = dd_ldexp(two_prod(x, x), -2);              /* x^2 / 4, exact */
  /* peak index: positive root of k (k + v) = x^2 / 4 (paper Eq. "K") */
  double vd = dd_to_d(v);
  double kpk = floor(0.5 * (-vd + hypot(vd, x)) + 0.5);
  if (kpk < 0.0) kpk = 0.0;
  /* L* = k* log(x^2/4) - lgamma(k*+1) - lgamma(k*+v+1) */
  dd lstar = dd_neg(dd_add(dd_lgamma(dd_from(kpk + 1.0)), dd_lgamma(dd_add_d(v, kpk + 1.0))));
  if (kpk > 0.0) lstar = dd_add(lstar, dd_mul_d(dd_log(y), kpk));
  /* T = sum over k != k* of a_k / a_{k*} (each positive) */
  dd T = dd_from(0.0);
  dd t = dd_from(1.0);
  for (double k = kpk + 1.0;; k += 1.0) {             /* forward */
    dd den = dd_mul_d(dd_add_d(v, k), k);
    t = dd_mul(t, dd_div(y, den));
    T = dd_add(T, t);
    if (t.hi < tiny * (1.0 + T.hi)) break;
  }
  t = dd_from(1.0);
  for (double k = kpk; k >= 1.0; k -= 1.0) {          /* backward: a_{k-1}/a_k = k(k+v)/y */
    dd num = dd_mul_d(dd_add_d(v, k), k);
    t = dd_mul(t, dd_div(num, y));
    T = dd_add(T, t);
    if (t.hi < tiny * (1.0 + T.hi)) break;
  }
  dd res = dd_add(lstar, dd_log1p(T));
  if (vd != 0.0) res = dd_add(res, dd_mul(v, dd_log(dd_from(0.5 * x))));
  return res;
}

/* ------------------------------------------------------------------ */
/* log K_v(x): trapezoid rule on int_0^inf exp(-x cosh t) cosh(v t) dt */
/* ------------------------------------------------------------------ */
/* phi(t) = -x cosh t + log cosh(v t), t >= 0 in double-double */
static dd k_phi(dd v, double x, dd t) {
  dd et = dd_exp(t);
  if (isinf(et.hi)) return dd_from(-INFINITY);        /* x cosh t overflows: the integrand is 0 */
  dd cosh_t = dd_ldexp(dd_add(et, dd_div(dd_from(1.0), et)), -1);
  dd a = dd_mul(v, t);                                /* v t >= 0 */
  /* log cosh a = a - ln 2 + log1p(exp(-2a)) */
  dd lc = dd_add(dd_sub(a, DD_LN2), dd_log1p(dd_exp(dd_ldexp(dd_neg(a), 1))));
  return dd_sub(lc, dd_mul_d(cosh_t, x));
}

/* exp(phi(t) - phi_max); 0 where x cosh t overflows (double-double
 * arithmetic on infinities would give NaN) */
static dd k_term(dd v, double x, dd t, dd pmax) {
  dd ph = k_phi(v, x, t);
  if (isinf(ph.hi)) return dd_from(0.0);
  return dd_exp(dd_sub(ph, pmax));
}

/* derivative of phi in plain double, used only to locate the peak */
static double k_dphi(double v, double x, double t) { return -x * sinh(t) + v * tanh(v * t); }

static dd log_k_dd(dd v, double x) {
  double vd = dd_to_d(v);
  /* peak t*: phi is unimodal on [0, inf); t* = 0 iff v^2 <= x */
  double ts = 0.0;
  if (vd * vd > x) {
    double lo = 0.0, hi = asinh(vd / x) + 1e-3;
    while (k_dphi(vd, x, hi) > 0.0) hi *= 2.0;
    for (int i = 0; i < 200 && hi - lo > 1e-15 * hi; ++i) {
      double mid = 0.5 * (lo + hi);
      if (k_dphi(vd, x, mid) > 0.0) lo = mid; else hi = mid;
    }
    ts = 0.5 * (lo + hi);
  }
  dd pmax = k_phi(v, x, dd_from(ts));
  /* curvature scale for the bracket search */
  double curv = x * cosh(ts) - vd * vd / (cosh(vd * ts) * cosh(vd * ts));
  double sig = 1.0 / sqrt(fabs(curv) + 1e-300);
  if (!(sig < 1.0)) sig = 1.0;
  const double drop = 90.0;                           /* exp(-90) ~ 8e-40 */
  double d = sig;
  while (dd_to_d(dd_sub(k_phi(v, x, dd_from(ts + d)), pmax)) > -drop) d *= 1.5;
  double thi = ts + d;
  double tlo = 0.0;
  if (ts > 0.0) {
    d = sig;
    while (ts - d > 0.0 && dd_to_d(dd_sub(k_phi(v, x, dd_from(ts - d)), pmax)) > -drop) d *= 1.5;
    tlo = ts - d > 0.0 ? ts - d : 0.0;
  }
  /* Trapezoid with step halving; nodes t_j = tlo + j h formed exactly in dd.
   * When tlo = 0 the integrand is even about 0, so the one-sided rule with
   * half weight at 0 is half the bi-infinite trapezoid rule. */
  int m = 64;
  double h = (thi - tlo) / m;
  dd sum = dd_from(0.0);
  for (int j = 0; j <= m; ++j) {
    dd tj = dd_add(dd_from(tlo), two_prod((double)j, h));
    dd f = k_term(v, x, tj, pmax);
    if (j == 0 || j == m) f = dd_ldexp(f, -1);
    sum = dd_add(sum, f);
  }
  dd est = dd_mul_d(sum, h);
  /* The trapezoid error for an analytic integrand behaves like exp(-c/h), so
   * each halving roughly squares it: once a halving changes the sum by less
   * than 1e-18 (relative), the new sum is accurate far beyond 1e-30.  The
   * double-double noise floor of phi where the integrand matters
   * (|x cosh t| <= |phi_max| + 90 + v t there) bounds what can be resolved. */
  double noise = ORACLE_NOISE_UNIT * (1.0 + fabs((double)pmax.hi) + 100.0 + 2.0 * vd * thi);
  if (noise < 1e-18) noise = 1e-18;
  for (int level = 0; level < 16; ++level) {
    dd add = dd_from(0.0);
    for (int j = 0; j < m; ++j) {
      dd tj = dd_add(dd_from(tlo), two_prod((double)j + 0.5, h));
      add = dd_add(add, k_term(v, x, tj, pmax));
    }
    sum = dd_add(sum, add);
    m *= 2;
    h *= 0.5;
    dd nest = dd_mul_d(sum, h);
    double change = fabs(dd_to_d(dd_sub(nest, est)));
    est = nest;
    if (level >= 1 && change < noise * est.hi) break;
  }
  return dd_add(pmax, dd_log(est));
}

/* ------------------------------------------------------------------ */
/* scalar entry points with the domain conventions                     */
/* ------------------------------------------------------------------ */
static dd special_i(double v, double x, int* done) {
  *done = 1;
  if (isnan(v) || isnan(x) || v < 0.0 || x < 0.0) return dd_from(NAN);
  if (isinf(v) && isinf(x)) return dd_from(NAN);
  if (isinf(x)) return dd_from(INFINITY);
  if (isinf(v)) return dd_from(-INFINITY);
  if (x == 0.0) return dd_from(v == 0.0 ? 0.0 : -INFINITY);
  *done = 0;
  return dd_from(0.0);
}
static dd special_k(double v, double x, int* done) {
  *done = 1;
  if (isnan(v) || isnan(x) || x < 0.0) return dd_from(NAN);
  if (isinf(v) && isinf(x)) return dd_from(NAN);
  if (isinf(x)) return dd_from(-INFINITY);
  if (x == 0.0 || isinf(v)) return dd_from(INFINITY);
  *done = 0;
  return dd_from(0.0);
}

/* The series needs O(sqrt(x)) terms around its peak; beyond this argument
 * the oracle declines (returns NaN) rather than run for hours. */
#define ORACLE_I_XMAX 1e8

static dd oracle_log_i_1(double v, double x) {
  int done; dd s = special_i(v, x, &done);
  if (done) return s;
  if (x > ORACLE_I_XMAX) return dd_from(NAN);
  return log_i_dd(dd_from(v), x);
}
static dd oracle_log_k_1(double v, double x) {
  int done; dd s = special_k(v, x, &done);
  return done ? s : log_k_dd(dd_from(fabs(v)), x);
}
/* d/dx log I_v = I_{v+1}/I_v + v/x */
static double oracle_dlog_i_1(double v, double x) {
  if (isnan(v) || isnan(x) || v < 0.0 || x < 0.0 || isinf(v) || isinf(x) || x > ORACLE_I_XMAX) return NAN;
  if (x == 0.0) return v == 0.0 ? 0.0 : INFINITY;   /* I_v ~ (x/2)^v / Gamma(v+1) */
  dd vv = dd_from(v);
  dd r = dd_exp(dd_sub(log_i_dd(dd_add_d(vv, 1.0), x), log_i_dd(vv, x)));
  return dd_to_d(dd_add(r, dd_div(vv, dd_from(x))));
}
/* d/dx log K_v = -(K_{v-1}/K_v + v/x), K_{v-1} = K_{|v-1|} */
static double oracle_dlog_k_1(double v, double x) {
  if (isnan(v) || isnan(x) || x <= 0.0 || isinf(v) || isinf(x)) return x == 0.0 ? -INFINITY : NAN;
  dd vv = dd_from(fabs(v));
  dd vm1 = dd_add_d(vv, -1.0);
  if (vm1.hi < 0.0) vm1 = dd_neg(vm1);
  dd r = dd_exp(dd_sub(log_k_dd(vm1, x), log_k_dd(vv, x)));
  return -dd_to_d(dd_add(r, dd_div(vv, dd_from(x))));
}
/* d/dv by a central difference of double-double values (used only to scale
 * the error metric; relative accuracy ~1e-10 is plenty). */
static double oracle_dlog_dv_1(int kind, double v, double x) {
  double h = 1e-6 * (fabs(v) > 1.0 ? fabs(v) : 1.0);
  if (!isfinite(v) || !isfinite(x) || x <= 0.0) return NAN;
  if (kind == 0) {
    if (x > ORACLE_I_XMAX) return NAN;
    if (v < 0.0) return NAN;
    double lo = v - h > 0.0 ? v - h : v, hi = v + h;
    dd f1 = log_i_dd(dd_from(hi), x), f0 = log_i_dd(dd_from(lo), x);
    return dd_to_d(dd_sub(f1, f0)) / (hi - lo);
  } else {
    double av = fabs(v);
    double lo = av - h, hi = av + h;
    dd f1 = log_k_dd(dd_from(fabs(hi)), x), f0 = log_k_dd(dd_from(fabs(lo)), x);
    double d = dd_to_d(dd_sub(f1, f0)) / (hi - lo);
    return v < 0.0 ? -d : d;
  }
}
/* vMF log-normaliser log C_d(k) = (d/2-1) log k - (d/2) log(2 pi) - log I_{d/2-1}(k) */
static double oracle_vmf_log_c_1(double d, double kappa) {
  if (isnan(kappa) || kappa < 0.0 || !(d >= 2.0) || kappa > ORACLE_I_XMAX) return NAN;
  if (kappa == 0.0) {
    /* limit: I_nu(k) ~ (k/2)^nu / Gamma(nu+1), so log C = -log(2) - (d/2) log(pi) + lgamma(d/2) */
    dd nu1 = dd_from(0.5 * d);
    dd r = dd_sub(dd_lgamma(nu1), dd_mul_d(dd_log(DD_PI), 0.5 * d));
    return dd_to_d(dd_sub(r, DD_LN2));
  }
  dd nu = dd_from(0.5 * d - 1.0);
  dd r = dd_mul(nu, dd_log(dd_from(kappa)));
  r = dd_sub(r, dd_mul_d(dd_log(dd_ldexp(DD_PI, 1)), 0.5 * d));
  r = dd_sub(r, log_i_dd(nu, kappa));
  return dd_to_d(r);
}

/* ------------------------------------------------------------------ */
/* threaded array drivers                                              */
/* ------------------------------------------------------------------ */
enum { OP_LOG_I = 0, OP_LOG_K = 1, OP_DLOG_I = 2, OP_DLOG_K = 3, OP_DV_I = 4, OP_DV_K = 5, OP_VMF = 6 };

typedef struct {
  int op, nthreads, tid;
  const double *v, *x;
  double *out, *out_lo;
  int64_t n;
} job_t;

static void* worker(void* arg) {
  job_t* j = (job_t*)arg;
  for (int64_t i = j->tid; i < j->n; i += j->nthreads) {
    double v = j->v[i], x = j->x[i];
    dd r;
    switch (j->op) {
      case OP_LOG_I: r = oracle_log_i_1(v, x); break;
      case OP_LOG_K: r = oracle_log_k_1(v, x); break;
      case OP_DLOG_I: r = dd_from(oracle_dlog_i_1(v, x)); break;
      case OP_DLOG_K: r = dd_from(oracle_dlog_k_1(v, x)); break;
      case OP_DV_I: r = dd_from(oracle_dlog_dv_1(0, v, x)); break;
      case OP_DV_K: r = dd_from(oracle_dlog_dv_1(1, v, x)); break;
      default: r = dd_from(oracle_vmf_log_c_1(v, x)); break;
    }
    double hi = r.hi + r.lo;
    j->out[i] = hi;
    if (j->out_lo) j->out_lo[i] = isfinite(hi) ? (r.hi - hi) + r.lo : 0.0;
  }
  return NULL;
}

/* Evaluate op over n (v, x) pairs with nthreads POSIX threads.  out receives
 * the double-double value rounded to double; out_lo (may be NULL) receives
 * the remainder, so out + out_lo carries ~106 bits.  For OP_VMF, v holds the
 * dimension d and x holds kappa.  Returns 0, or -1 on a thread error. */
int oracle_eval(int op, const double* v, const double* x, double* out, double* out_lo, int64_t n,
                int nthreads) {
  init_tables();
  if (n <= 0) return 0;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = (int)n;
  pthread_t th[256];
  job_t jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (job_t){op, nthreads, t, v, x, out, out_lo, n};
    if (t > 0 && pthread_create(&th[t], NULL, worker, &jobs[t]) != 0) return -1;
  }
  worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* Exposed double-double primitives, so the test suite can pin them one by
 * one against exact or arbitrary-precision values. */
void oracle_dd_exp(double hi, double lo, double* out2) { init_tables(); dd r = dd_exp(dd_make(hi, lo)); out2[0] = r.hi; out2[1] = r.lo; }
void oracle_dd_log(double hi, double lo, double* out2) { init_tables(); dd r = dd_log(dd_make(hi, lo)); out2[0] = r.hi; out2[1] = r.lo; }
void oracle_dd_lgamma(double hi, double lo, double* out2) { init_tables(); dd r = dd_lgamma(dd_make(hi, lo)); out2[0] = r.hi; out2[1] = r.lo; }
void oracle_dd_log1p(double hi, double lo, double* out2) { init_tables(); dd r = dd_log1p(dd_make(hi, lo)); out2[0] = r.hi; out2[1] = r.lo; }
void oracle_dd_const(int which, double* out2) {
  dd r = which == 0 ? DD_LN2 : DD_PI;
  out2[0] = r.hi; out2[1] = r.lo;
}

/* Significand bits of the arithmetic this build evaluates in: 106 for
 * double-double (two 53-bit doubles), LDBL_MANT_DIG for the long double build. */
int oracle_significand_bits(void) {
#ifdef ORACLE_LONG_DOUBLE
  return LDBL_MANT_DIG;
#else
  return 106;
#endif
}
