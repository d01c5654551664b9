"""Algorithmic FP64 work of the evaluation kernels, for roofline reporting.

Work is counted in FP64 pipe slots: one slot per double add, multiply or fused
multiply-add the method performs, and for each library call (exp, log,
lgamma, division, square root) the number of DFMA issue slots that one call
occupies on this GPU, i.e. (DFMA throughput) / (call throughput), both
measured with all SMs busy by the microbenchmarks of fp64_peak.cu.  FLOPs are
reported as 2 x slots (an FMA counts two).

The counts follow the expressions as written in lb_expr.cuh and lb_kint.cuh;
they are the method's arithmetic, not the instructions a profiler counts.
"""
import numpy as np

# DFMA-slot cost of one call, from the measured throughput ratios on GB300
# (DFMA 0.597 T/s; exp 31.4 G/s, log 17.1 G/s, div 58.2 G/s, sqrt 58.1 G/s,
# lgamma 20.7 G/s on arguments 2..4).
SLOT_EXP = 19.0
SLOT_LOG = 34.9
SLOT_DIV = 10.3
SLOT_SQRT = 10.3
SLOT_LGAMMA = 28.9


def kint_rule(v, x):
    """Node counts (g, h) of the tight K-integral rule for each pair (|v| given)."""
    v = np.asarray(v, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    ng = np.where((v >= 0.9) | (x >= 0.25), 32, np.where((v >= 0.4) | (x >= 1e-3), 64, 128))
    nh = np.where(v <= 1.2, 32, np.where(v <= 5.0, 48, 32))
    return ng, nh


def kint_slots(v, x):
    """FP64 slots of one K-integral evaluation per pair (tight Gauss rule)."""
    ng, nh = kint_rule(v, x)
    # g node: beta*log u, exp, 3 adds, log, (v-1/2)*log + 7 log u (mul + fma),
    #         then exp(L - m): subtract, exp, accumulate
    g_node = 1 + SLOT_EXP + 3 + SLOT_LOG + 2 + 1 + SLOT_EXP + 1
    # h node: s + 2x, log, + y, fma, then subtract, exp, accumulate
    h_node = 1 + SLOT_LOG + 1 + 1 + 1 + SLOT_EXP + 1
    # per pair: beta (div), log beta, 2 small ops, final log and adds, the
    # warp reductions (5 adds), and the prefactor (lgamma, log, 3 ops)
    per_pair = SLOT_DIV + SLOT_LOG + 2 + SLOT_LOG + 2 + 5 + SLOT_LGAMMA + SLOT_LOG + 3
    return ng * g_node + nh * h_node + per_pair


def mu20_slots():
    # 20 terms: subtract, two multiplies, one fma; plus 1/(8x), rsqrt/sqrt, product, log, add
    return 20 * 4 + SLOT_DIV + SLOT_SQRT + 2 + SLOT_LOG + 1


def u13_slots():
    # x/v, fma+sqrt, 1/r, t*t, t/v, 91 Horner fmas of P_k + 13 in q, eta (add, div, log, add),
    # tail (multiplies, rsqrt, log, fma)
    return (SLOT_DIV + 1 + SLOT_SQRT + SLOT_DIV + 1 + SLOT_DIV + 91 + 13
            + 1 + SLOT_DIV + SLOT_LOG + 1 + 3 + SLOT_SQRT + SLOT_LOG + 1)


def series_terms(v, x):
    """Number of series terms the I fallback sums for each pair (same stopping rule)."""
    v = np.asarray(v, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    y = 0.25 * x * x
    kpk = 0.5 * (np.sqrt(x * x + v * v) - v)
    term = np.ones_like(x)
    T = np.zeros_like(x)
    done = np.zeros(x.shape, dtype=bool)
    count = np.zeros(x.shape, dtype=np.int64)
    k = 1.0
    for _ in range(400):
        active = ~done
        if not active.any():
            break
        term = np.where(active, term * y / (k * (k + v)), term)
        T = np.where(active, T + term, T)
        count += active
        done |= active & (k > kpk) & (term <= 1.3877787807814457e-17 * (1.0 + T))
        k += 1.0
    return count


def series_slots(v, x):
    # per term: divide, 2 multiplies/adds for k(k+v), multiply, add; plus sqrt for the
    # peak, lgamma, log1p, log, fma
    n = series_terms(v, x)
    return n * (SLOT_DIV + 4) + SLOT_SQRT + 3 + SLOT_LGAMMA + SLOT_LOG + SLOT_LOG + 2
