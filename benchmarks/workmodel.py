"""Algorithmic FP64 work of the evaluation kernels, for roofline reporting.

Work is counted in FP64 pipe slots: one slot per double add, multiply, fused
multiply-add or compare the method performs, and for each library call
(division, square root, reciprocal square root, lgamma) the number of DFMA
issue slots one call occupies on this GPU, i.e. (DFMA throughput) / (call
throughput) less the one extra operation of the measuring loop, both
measured with all SMs busy by logbessel_measure_fp64.  The table-driven exp
and log of lb_fastmath.cuh and the integer-pipe exp, log, reciprocal and
1/sqrt of lb_intmath.cuh are counted the same way.
FLOP = 2 x slots (an FMA counts two).

The counts follow the code paths of lb_expr.cuh and lb_kint.cuh (tight mode,
FP64).  The exps and logs of the K-integral nodes run on the integer pipes
(lb_intmath.cuh); they are priced by the same measured rule, so the sum of
slots is the time the kernel's operations would take one after another at
full throughput, and frac = that time / the measured time.  Term counts are the per-pair counts of the single-precision pre-pass;
the kernels run the maximum over each warp, so the real work is slightly
higher than counted here.
"""
import numpy as np

# DFMA-slot cost of one call: (DFMA rate) / (call rate) - 1, the rates measured
# with all SMs busy by logbessel_measure_fp64 (the 1 is the extra operation per
# call of its throughput loop).  These defaults are one GB300 measurement
# (DFMA 627 G/s; division 61.2, sqrt 61.1, lgamma 21.9 G/s); bench.py replaces
# them with the rates it measures on the GPU it runs on (set_costs).
SLOT_DIV = 9.2
SLOT_SQRT = 9.3
SLOT_RSQRT = 9.3
SLOT_LGAMMA = 27.6
# table-driven exp/log of lb_fastmath.cuh: 10, 9 and 14 FP64 operations as
# written; the measured costs replace these
SLOT_EXP = 10.0
SLOT_EXP_TERM = 9.0
SLOT_LOG = 14.0
# exp and log on the integer pipes (lb_intmath.cuh), priced the same way: the
# DFMA slots that the time of one call at full throughput would hold
SLOT_IX_EXP = 3.0
SLOT_IX_LOG = 3.5
# reciprocal and 1/sqrt on the integer pipes (lb_intmath.cuh), priced the same way
SLOT_IX_RCP = 3.5
SLOT_IX_RSQRT = 4.0


def set_costs(rates):
    """Set the slot costs from measured rates (dict of operations per second,
    as returned by _binding.measure_fp64)."""
    global SLOT_DIV, SLOT_SQRT, SLOT_RSQRT, SLOT_LGAMMA, SLOT_EXP, SLOT_EXP_TERM, SLOT_LOG, SLOT_IX_EXP, SLOT_IX_LOG
    global SLOT_IX_RCP, SLOT_IX_RSQRT
    d = rates["dfma"]
    SLOT_DIV = d / rates["div"] - 1.0
    SLOT_SQRT = SLOT_RSQRT = d / rates["sqrt"] - 1.0
    SLOT_LGAMMA = d / rates["lgamma"] - 1.0
    SLOT_EXP = d / rates["fm_exp"] - 1.0
    SLOT_LOG = d / rates["fm_log"] - 1.0
    if "fm_exp_term" in rates:
        SLOT_EXP_TERM = d / rates["fm_exp_term"] - 1.0
    if "ix_exp" in rates:
        SLOT_IX_EXP = d / rates["ix_exp"] - 1.0
        SLOT_IX_LOG = d / rates["ix_log"] - 1.0
    if "ix_rcp" in rates:
        SLOT_IX_RCP = d / rates["ix_rcp"] - 1.0
        SLOT_IX_RSQRT = d / rates["ix_rsqrt"] - 1.0
    return {"div": SLOT_DIV, "sqrt": SLOT_SQRT, "lgamma": SLOT_LGAMMA, "fm_exp": SLOT_EXP,
            "fm_exp_term": SLOT_EXP_TERM, "fm_log": SLOT_LOG, "ix_exp": SLOT_IX_EXP, "ix_log": SLOT_IX_LOG,
            "ix_rcp": SLOT_IX_RCP, "ix_rsqrt": SLOT_IX_RSQRT}


REGION_K = {0: 20, 1: 13, 4: 3, 5: 4, 6: 6, 7: 9}   # region id -> number of expansion terms


def kint_rule(v, x, dx=False):
    """Node counts (g, h) of the tight K-integral rule for each pair (|v| given).
    The split g rule (v < 0.4, x < 1e-3) has 64 + 32 + 32 nodes, plus 32 more
    below x ~ 4e-21; for 1.2 < v <= 5 the rule is 24 g + 40 h nodes; values
    (dx False) with 2 <= v <= 16.5 take the one-slot rules, 22 + 10 nodes
    (v < 7) or 12 + 20."""
    v = np.asarray(v, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    split = np.where(np.log(128 * np.maximum(x, 1e-320)) + 40 < -4, 160, 128)
    ng = np.where((v >= 0.9) | (x >= 0.25), 32, np.where((v >= 0.4) | (x >= 1e-3), 64, split))
    nh = np.where(v <= 1.2, 32, np.where(v <= 5.0, 48, 32))
    packed = (v > 1.2) & (v <= 5.0)                 # 24 g + 40 h nodes
    ng, nh = np.where(packed, 24, ng), np.where(packed, 40, nh)
    if not dx:
        one = (v >= 2.0) & (v <= 16.5)
        ng = np.where(one, np.where(v < 7.0, 22, 12), ng)
        nh = np.where(one, np.where(v < 7.0, 10, 20), nh)
    return ng, nh


def kint_slots(v, x, scalar=False):
    """Work of one K-integral evaluation per pair (tight Gauss rule), in DFMA
    slots; the node exps and logs are the integer-pipe ones.  scalar=True for
    a call with one order for all pairs (node positions u^beta and lgamma
    computed once per block)."""
    ng, nh = kint_rule(v, x)
    split = ng > 64
    # g node: beta*log u (+ log s0), exp, 2x + s, log, c + log beta, fma, - s;
    # then L - m and the exp (the sum is formed in fixed point on the integer
    # pipe; the split rule adds in FP64 and has 3 more for its offset form)
    g_node = (5 if scalar else 6 + SLOT_IX_EXP) + SLOT_IX_EXP + SLOT_IX_LOG + np.where(split, 4, 0)
    # h node: s + 2x, log, + y, fma; then L - m, exp (split rule: + 1 add)
    h_node = 4 + SLOT_IX_EXP + SLOT_IX_LOG + np.where(split, 1, 0)
    # per pair (once per lane of its batch): beta (reciprocal, 2 ops), lgamma,
    # prefactor (log, 3 ops), log beta (+ fma), final log and add, the fixed
    # sum to double (2 ops)
    per_pair = SLOT_IX_RCP + 2 + (0 if scalar else SLOT_LGAMMA) + SLOT_IX_LOG + 3 + SLOT_IX_LOG + 2 + SLOT_IX_LOG + 1 + 2
    # split rule: log s1, C, three panel widths (log + add each), the flat
    # term (log, expm1, division), its FP64 warp sum (5 adds)
    per_pair = per_pair + np.where(split, 2 + 4 * SLOT_LOG + 3 + SLOT_EXP + SLOT_DIV + 4 + 5, 0)
    return ng * g_node + nh * h_node + per_pair


def mu_terms(v, x, K=20):
    """Terms summed by the mu_K expression (single-precision pre-pass rule)."""
    v = np.asarray(v, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    mu = 4.0 * v * v
    inv8x = np.float32(1.0) / (np.float32(8.0) * x)
    t = np.ones_like(x)
    n = np.full(x.shape, K, dtype=np.int64)
    done = np.zeros(x.shape, dtype=bool)
    for k in range(1, K + 1):
        t = np.where(done, t, t * (mu - np.float32((2 * k - 1) ** 2)) * inv8x / np.float32(k))
        hit = ~done & (np.abs(t) < 1.4e-17)
        n = np.where(hit, k, n)
        done |= hit
    return n


def mu_slots(v, x, K=20):
    # per term: fma, multiply, fma; plus 4v^2, 1/(8x), S^2 and two products, log, fma
    return mu_terms(v, x, K) * 3 + 2 + SLOT_IX_RCP + 4 + SLOT_IX_LOG + 1


def u_slots(K):
    # 1/v, x/v, fma, rsqrt, r = r2 t, t*t, t/v, sum_k k Horner fmas of P_k, K in q,
    # eta (add, two logs, subtract, add), tail (3 multiplies, log, 2 multiplies, fma)
    horner = sum(k for k in range(1, K + 1)) + K
    return (SLOT_IX_RCP + 1 + 1 + SLOT_IX_RSQRT + 1 + 1 + 1 + horner
            + 1 + 2 * SLOT_IX_LOG + 1 + 1 + 3 + SLOT_IX_LOG + 3)


def series_terms(v, x):
    """Terms the I power series sums for each pair (single-precision pre-pass rule)."""
    v = np.asarray(v, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    y = np.float32(0.25) * x * x
    kpk = np.float32(0.5) * (np.sqrt(x * x + v * v) - v)
    term = np.ones_like(x)
    T = np.zeros_like(x)
    n = np.ones(x.shape, dtype=np.int64)
    done = np.zeros(x.shape, dtype=bool)
    for k in range(1, 91):
        active = ~done
        if not active.any():
            break
        term = np.where(active, term * y / (np.float32(k) * (np.float32(k) + v)), term)
        T = np.where(active, T + term, T)
        n = np.where(active, k, n)
        done |= active & (np.float32(k) > kpk) & (term <= np.float32(1.4e-17) * (1 + T))
    return n


def series_slots(v, x):
    # per term: d = k v + k^2 (fma), y A, fma, B d; plus A/B, log, lgamma, log(x/2), fma
    n = series_terms(v, x)
    return n * 4 + SLOT_IX_RCP + 1 + SLOT_IX_LOG + SLOT_LGAMMA + SLOT_IX_LOG + 3


def mu_slots_scalar(v, x, K=20):
    # one order for all pairs: per term one fma; plus 1/(8x), S^2 and two products, log, fma
    return mu_terms(v, x, K) * 1 + SLOT_IX_RCP + 1 + 3 + SLOT_IX_LOG + 1


def u_slots_scalar(K):
    # x/v, fma, rsqrt, r2 t, Horner of degree 3K in t, eta (add, two logs, subtract, add),
    # tail (3 multiplies, log, 2 multiplies, fma)
    return 1 + 1 + SLOT_IX_RSQRT + 1 + 3 * K + 1 + 2 * SLOT_IX_LOG + 1 + 1 + 3 + SLOT_IX_LOG + 3


def series_slots_scalar(v, x):
    # per term: y r_k, fma; plus y, log P, log(x/2), fma
    n = series_terms(v, x)
    return n * 2 + 2 + SLOT_IX_LOG + SLOT_IX_LOG + 3


def region_slots(region, v, x, scalar=False):
    """FP64 slots of the per-thread expressions (tiles kernel) for pairs of one
    region; scalar=True for a call with one order for all pairs (the order's
    constants are computed once per block, see ScalarOrder)."""
    if region == 0:
        return mu_slots_scalar(v, x) if scalar else mu_slots(v, x)
    if region in REGION_K and region != 4:
        k = REGION_K[region]
        return np.full(np.shape(x), u_slots_scalar(k) if scalar else u_slots(k), dtype=np.float64)
    if region == 4:
        return mu_slots(v, x, K=3)
    return series_slots_scalar(v, x) if scalar else series_slots(v, x)
